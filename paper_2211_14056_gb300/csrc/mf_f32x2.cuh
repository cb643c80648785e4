// Packed FP32 pairs for the amplitude kernel: f2 holds the same quantity for
// two independent evaluations (here the two antitop helicities of a lane), and
// its arithmetic issues Blackwell's paired FP32 instructions (one instruction
// for both halves, each half rounded exactly as the scalar operation).  The
// amplitude kernel is bound by instruction issue, not by the FMA pipes, so
// halving the FP32 instruction count of its quark-line walk shortens it.
#pragma once
#include <cuda_runtime.h>

#include "mf_device.cuh"

namespace mf {

struct f2 {
  float2 v;
  __device__ __forceinline__ f2() {}
  __device__ __forceinline__ explicit f2(float s) : v(make_float2(s, s)) {}
  __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
};

__device__ __forceinline__ f2 operator+(f2 a, f2 b) { f2 o; o.v = __fadd2_rn(a.v, b.v); return o; }
__device__ __forceinline__ f2 operator-(f2 a) { return f2(-a.v.x, -a.v.y); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { f2 o; o.v = __fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y)); return o; }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { f2 o; o.v = __fmul2_rn(a.v, b.v); return o; }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) { f2 o; o.v = __ffma2_rn(a.v, b.v, c.v); return o; }

// both halves from one scalar quantity
__device__ __forceinline__ cplx<f2> dup(cplx<float> a) { return {f2(a.r), f2(a.i)}; }
__device__ __forceinline__ R4<f2> dup(const R4<float>& a) {
  return {{f2(a.v[0]), f2(a.v[1]), f2(a.v[2]), f2(a.v[3])}};
}
__device__ __forceinline__ Slash<f2> dup(const Slash<float>& s) { return {dup(s.a), dup(s.b), dup(s.c), dup(s.d)}; }
// one half from each of two scalar quantities
__device__ __forceinline__ cplx<f2> pack(cplx<float> a, cplx<float> b) { return {f2(a.r, b.r), f2(a.i, b.i)}; }
__device__ __forceinline__ S4<f2> pack(const S4<float>& a, const S4<float>& b) {
  S4<f2> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.c[k] = pack(a.c[k], b.c[k]);
  return o;
}

// row spinor (the same for both halves) times a packed column spinor
__device__ __forceinline__ cplx<f2> rowdot(const S4<float>& row, const S4<f2>& col) {
  const cplx<f2> a = cfma(dup(row.c[1]), col.c[1], dup(row.c[0]) * col.c[0]);
  const cplx<f2> b = cfma(dup(row.c[3]), col.c[3], dup(row.c[2]) * col.c[2]);
  return a + b;
}

}  // namespace mf
