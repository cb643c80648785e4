// Forward-mode dual numbers for the derivative kernels: a value and N
// tangents, with the chain rule for every operation the sampling and
// amplitude code uses.  The value parts call the ordinary CUDA math
// functions; the tangents follow from the derivatives of those functions.
//
// The derivative of the event weight with respect to g_s, m_t, Gamma_t and the
// Vegas uniforms (arXiv:2211.14056, Sec. 2: the custom operator lacks a
// derivative, "trivial to extend") is obtained by running the same templated
// code with T = Dual<B, N>: every wavefunction, current and amplitude is
// recomputed with its tangents, nothing is stored between passes.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>

namespace mf {

// the ordinary math functions stay visible next to the dual overloads below
using ::acos;
using ::atan2;
using ::cos;
using ::exp;
using ::expm1;
using ::fabs;
using ::fma;
using ::fmax;
using ::log;
using ::log1p;
using ::rsqrt;
using ::sqrt;

template <typename B, int N> struct Dual {
  B v;
  B d[N];
  __host__ __device__ Dual() {}
  __host__ __device__ Dual(B x) : v(x) {
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = B(0);
  }
  template <typename A, typename = typename std::enable_if<std::is_arithmetic<A>::value && !std::is_same<A, B>::value>::type>
  __host__ __device__ Dual(A x) : Dual(B(x)) {}
  template <typename C, typename = typename std::enable_if<!std::is_same<C, B>::value>::type>
  __host__ __device__ explicit Dual(const Dual<C, N>& o) : v(B(o.v)) {
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = B(o.d[k]);
  }
  __host__ __device__ explicit operator B() const { return v; }
};

template <typename X> struct is_dual { static constexpr bool value = false; };
template <typename B, int N> struct is_dual<Dual<B, N>> { static constexpr bool value = true; };

template <typename X> __host__ __device__ __forceinline__ X value_of(X x) { return x; }
template <typename B, int N> __host__ __device__ __forceinline__ B value_of(const Dual<B, N>& x) { return x.v; }

#define MF_D(B, N) Dual<B, N>

template <typename B, int N>
__host__ __device__ __forceinline__ Dual<B, N> operator+(const Dual<B, N>& a, const Dual<B, N>& b) {
  Dual<B, N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <typename B, int N>
__host__ __device__ __forceinline__ Dual<B, N> operator-(const Dual<B, N>& a, const Dual<B, N>& b) {
  Dual<B, N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <typename B, int N> __host__ __device__ __forceinline__ Dual<B, N> operator-(const Dual<B, N>& a) {
  Dual<B, N> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
  return r;
}
template <typename B, int N>
__host__ __device__ __forceinline__ Dual<B, N> operator*(const Dual<B, N>& a, const Dual<B, N>& b) {
  Dual<B, N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <typename B, int N>
__host__ __device__ __forceinline__ Dual<B, N> operator/(const Dual<B, N>& a, const Dual<B, N>& b) {
  Dual<B, N> r;
  const B ib = B(1) / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
// scalar on either side
#define MF_DUAL_SCALAR_OPS(OP)                                                                        \
  template <typename B, int N>                                                                        \
  __host__ __device__ __forceinline__ Dual<B, N> operator OP(const Dual<B, N>& a, B s) {              \
    return a OP Dual<B, N>(s);                                                                        \
  }                                                                                                   \
  template <typename B, int N>                                                                        \
  __host__ __device__ __forceinline__ Dual<B, N> operator OP(B s, const Dual<B, N>& a) {              \
    return Dual<B, N>(s) OP a;                                                                        \
  }
MF_DUAL_SCALAR_OPS(+)
MF_DUAL_SCALAR_OPS(-)
MF_DUAL_SCALAR_OPS(*)
MF_DUAL_SCALAR_OPS(/)
#undef MF_DUAL_SCALAR_OPS

template <typename B, int N> __host__ __device__ __forceinline__ Dual<B, N>& operator+=(Dual<B, N>& a, const Dual<B, N>& b) { a = a + b; return a; }
template <typename B, int N> __host__ __device__ __forceinline__ Dual<B, N>& operator-=(Dual<B, N>& a, const Dual<B, N>& b) { a = a - b; return a; }
template <typename B, int N> __host__ __device__ __forceinline__ Dual<B, N>& operator*=(Dual<B, N>& a, const Dual<B, N>& b) { a = a * b; return a; }

#define MF_DUAL_CMP(OP)                                                                                          \
  template <typename B, int N> __host__ __device__ __forceinline__ bool operator OP(const Dual<B, N>& a, const Dual<B, N>& b) { return a.v OP b.v; } \
  template <typename B, int N> __host__ __device__ __forceinline__ bool operator OP(const Dual<B, N>& a, B b) { return a.v OP b; }                   \
  template <typename B, int N> __host__ __device__ __forceinline__ bool operator OP(B a, const Dual<B, N>& b) { return a OP b.v; }
MF_DUAL_CMP(<)
MF_DUAL_CMP(>)
MF_DUAL_CMP(<=)
MF_DUAL_CMP(>=)
MF_DUAL_CMP(==)
#undef MF_DUAL_CMP

// f(a) with f'(a.v) = df
template <typename B, int N>
__host__ __device__ __forceinline__ Dual<B, N> chain(const Dual<B, N>& a, B f, B df) {
  Dual<B, N> r;
  r.v = f;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = df * a.d[k];
  return r;
}

template <typename B, int N>
__host__ __device__ __forceinline__ Dual<B, N> fma(const Dual<B, N>& a, const Dual<B, N>& b, const Dual<B, N>& c) {
  Dual<B, N> r;
  r.v = fma(a.v, b.v, c.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = fma(a.d[k], b.v, fma(a.v, b.d[k], c.d[k]));
  return r;
}
template <typename B, int N> __host__ __device__ __forceinline__ Dual<B, N> sqrt(const Dual<B, N>& a) {
  const B s = sqrt(a.v);
  return chain(a, s, s > B(0) ? B(0.5) / s : B(0));
}
template <typename B, int N> __host__ __device__ __forceinline__ Dual<B, N> rsqrt(const Dual<B, N>& a) {
  const B s = rsqrt(a.v);
  return chain(a, s, B(-0.5) * s * s * s);
}
template <typename B, int N> __host__ __device__ __forceinline__ Dual<B, N> exp(const Dual<B, N>& a) {
  const B e = exp(a.v);
  return chain(a, e, e);
}
template <typename B, int N> __host__ __device__ __forceinline__ Dual<B, N> log(const Dual<B, N>& a) {
  return chain(a, log(a.v), B(1) / a.v);
}
template <typename B, int N> __host__ __device__ __forceinline__ Dual<B, N> expm1(const Dual<B, N>& a) {
  return chain(a, expm1(a.v), exp(a.v));
}
template <typename B, int N> __host__ __device__ __forceinline__ Dual<B, N> log1p(const Dual<B, N>& a) {
  return chain(a, log1p(a.v), B(1) / (B(1) + a.v));
}
template <typename B, int N> __host__ __device__ __forceinline__ Dual<B, N> cos(const Dual<B, N>& a) {
  return chain(a, cos(a.v), -sin(a.v));
}
template <typename B, int N> __host__ __device__ __forceinline__ Dual<B, N> acos(const Dual<B, N>& a) {
  const B s = sqrt(B(1) - a.v * a.v);
  return chain(a, acos(a.v), s > B(0) ? B(-1) / s : B(0));
}
template <typename B, int N> __host__ __device__ __forceinline__ Dual<B, N> fabs(const Dual<B, N>& a) {
  return a.v < B(0) ? -a : a;
}
template <typename B, int N>
__host__ __device__ __forceinline__ Dual<B, N> fmax(const Dual<B, N>& a, const Dual<B, N>& b) {
  return a.v >= b.v ? a : b;
}
template <typename B, int N>
__host__ __device__ __forceinline__ Dual<B, N> atan2(const Dual<B, N>& y, const Dual<B, N>& x) {
  Dual<B, N> r;
  r.v = atan2(y.v, x.v);
  const B inv = B(1) / (x.v * x.v + y.v * y.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) * inv;
  return r;
}
// sin and cos of 2 pi t (t in turns)
template <typename B, int N>
__host__ __device__ __forceinline__ void sincos_turns(const Dual<B, N>& t, Dual<B, N>* s, Dual<B, N>* c) {
  B sv, cv;
  if constexpr (sizeof(B) == sizeof(float)) sincospif(B(2) * t.v, &sv, &cv);
  else sincospi(B(2) * t.v, &sv, &cv);
  const B w = B(6.283185307179586476925286766559);
  *s = chain(t, sv, w * cv);
  *c = chain(t, cv, -w * sv);
}

// warp shuffles of plain and dual values
template <typename X> __device__ __forceinline__ X shfl_any(unsigned mask, X x, int src) {
  return __shfl_sync(mask, x, src);
}
template <typename B, int N> __device__ __forceinline__ Dual<B, N> shfl_any(unsigned mask, const Dual<B, N>& x, int src) {
  Dual<B, N> r;
  r.v = __shfl_sync(mask, x.v, src);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = __shfl_sync(mask, x.d[k], src);
  return r;
}
template <typename X> __device__ __forceinline__ X shfl_xor_any(unsigned mask, X x, int off) {
  return __shfl_xor_sync(mask, x, off);
}
template <typename B, int N>
__device__ __forceinline__ Dual<B, N> shfl_xor_any(unsigned mask, const Dual<B, N>& x, int off) {
  Dual<B, N> r;
  r.v = __shfl_xor_sync(mask, x.v, off);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = __shfl_xor_sync(mask, x.d[k], off);
  return r;
}

}  // namespace mf
