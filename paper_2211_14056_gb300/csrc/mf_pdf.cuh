// Parton densities from a table: log-bicubic Hermite interpolation of
// x f(x, Q^2) (arXiv:2211.14056 Sec. 1: the integrand's densities come from
// PDFFlow, the GPU interpolation of tabulated LHAPDF sets).
//
// The scheme: on nodes uniform in ln x (step h_x) and ln Q^2 (step h_q), the
// ln x slope of a row's node is the finite difference of the row's values
// (mean of the two neighbouring quotients, one-sided at the first and last
// node); a query (x, Q^2), clamped to the table's range and located in cell
// (i, j) with local coordinates (u, v), is interpolated in ln x by a cubic
// Hermite polynomial on each row around it, and in ln Q^2 by a cubic Hermite
// step whose slopes at s_j and s_j+1 are the same finite differences of those
// row values.
//
// Stored form: per flavour and node (l, k) four numbers, every slope per unit
// of the local coordinate: f, df = FD_x(f), dq = FD_q(f) and dfq = FD_x(dq).
// Because the x-interpolation and the finite differences are linear, the ln Q^2
// slope at row l of the interpolated rows, FD_q(g)_l, equals the
// x-interpolation of (dq, dfq) on row l: a query reads two rows of two nodes
// (four 4-tuples), five Hermite steps, no branch at the table's edges.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mf {

constexpr int kMaxPdfPairs = 8;

// Device view of a loaded set: node tables in FP64 and FP32, flavour-major,
// node (l, k) of a flavour at 4 (l nx + k) (f, df, dq, dfq), each flavour's
// slice padded to `slice` elements.
struct PdfView {
  const double* tab64;
  const float* tab32;
  int nflav, nq, nx;
  int64_t slice;            // elements per flavour (>= nq * nx * 4)
  double t0, ht, s0, hs;    // ln x_min and the ln x step; ln Q2_min and the ln Q^2 step
  double iht, ihs;          // 1 / ht, 1 / hs
  float t0f, htf, s0f, ihtf, ihsf;   // the same in FP32 (no FP64 conversion per point in FP32)
};

template <typename K> struct PdfCell {
  int i, j;   // cell in ln x and ln Q^2
  K u, v;     // local coordinates in [0, 1]
};

template <typename K> __device__ __forceinline__ const K* pdf_table(const PdfView& pv);
template <> __device__ __forceinline__ const double* pdf_table<double>(const PdfView& pv) { return pv.tab64; }
template <> __device__ __forceinline__ const float* pdf_table<float>(const PdfView& pv) { return pv.tab32; }

// (cell, local coordinate) of a logarithm on n nodes c0 + k h (ih = 1/h), clamped to the range
template <typename K>
__device__ __forceinline__ void pdf_locate(K z, K c0, K ih, int n, int& cell, K& loc) {
  K r = (z - c0) * ih;
  r = r < K(0) ? K(0) : (r > K(n - 1) ? K(n - 1) : r);
  int k = int(r);
  k = k > n - 2 ? n - 2 : k;
  cell = k;
  loc = r - K(k);
}

__device__ __forceinline__ PdfCell<double> pdf_cell(const PdfView& pv, double lnx, double lnq2) {
  PdfCell<double> c;
  pdf_locate(lnx, pv.t0, pv.iht, pv.nx, c.i, c.u);
  pdf_locate(lnq2, pv.s0, pv.ihs, pv.nq, c.j, c.v);
  return c;
}
__device__ __forceinline__ PdfCell<float> pdf_cell(const PdfView& pv, float lnx, float lnq2) {
  PdfCell<float> c;
  pdf_locate(lnx, pv.t0f, pv.ihtf, pv.nx, c.i, c.u);
  pdf_locate(lnq2, pv.s0f, pv.ihsf, pv.nq, c.j, c.v);
  return c;
}

// ln x of an FP64 input in FP32 arithmetic without an FP64 instruction (an
// FP64 -> FP32 conversion issues on GB300's narrow FP64 pipe): x = 2^e m,
// m in [1, 2) rebuilt as an FP32 from the top 23 mantissa bits (relative
// error below 2^-23), ln x = (e + log2 m) ln 2.  x <= 0 or subnormal gives a
// large negative value (the callers clamp to the table).
__device__ __forceinline__ float log_f64_in_f32(double x) {
  const long long b = __double_as_longlong(x);
  const int e = int((b >> 52) & 0x7ff) - 1023;
  const float m = __int_as_float(0x3f800000 | int((b >> 29) & 0x7fffff));
  // log2 m by the special-function unit (absolute error ~2^-22 on [1, 2))
  return (float(e) + __log2f(m)) * 0.69314718055994531f;
}

// an FP32 value widened to FP64 with integer operations (zero for FP32
// subnormals, which no density here reaches)
__device__ __forceinline__ double widen_f32(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex == 0u) return __longlong_as_double((long long)(u & 0x80000000u) << 32);
  const unsigned long long e11 = ex == 0xffu ? 0x7ffull : (unsigned long long)(ex + 896u);
  const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) | (e11 << 52) |
                                  ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// cubic Hermite through (0, f0, slope d0) and (1, f1, slope d1), the slopes
// per unit of the local coordinate, in Horner form
template <typename K> __device__ __forceinline__ K hermite01(K w, K f0, K f1, K d0, K d1) {
  const K df = f1 - f0;
  const K c2 = K(3) * df - K(2) * d0 - d1;
  const K c3 = d0 + d1 - K(2) * df;
  return fma(w, fma(w, fma(w, c3, c2), d0), f0);
}

// x f(x, Q^2) of the flavour whose slice starts at `fl`
template <typename K>
__device__ __forceinline__ K pdf_xfx_slice(const PdfView& pv, const K* fl, const PdfCell<K>& c) {
  const K* a = fl + (int64_t(c.j) * pv.nx + c.i) * 4;   // row j: nodes i, i + 1
  const K* b = a + int64_t(pv.nx) * 4;                   // row j + 1
  K na[8], nb[8];
  if constexpr (sizeof(K) == sizeof(float)) {
    const float4 a0 = *reinterpret_cast<const float4*>(a), a1 = *reinterpret_cast<const float4*>(a + 4);
    const float4 b0 = *reinterpret_cast<const float4*>(b), b1 = *reinterpret_cast<const float4*>(b + 4);
    na[0] = a0.x; na[1] = a0.y; na[2] = a0.z; na[3] = a0.w; na[4] = a1.x; na[5] = a1.y; na[6] = a1.z; na[7] = a1.w;
    nb[0] = b0.x; nb[1] = b0.y; nb[2] = b0.z; nb[3] = b0.w; nb[4] = b1.x; nb[5] = b1.y; nb[6] = b1.z; nb[7] = b1.w;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double2 av = *reinterpret_cast<const double2*>(a + 2 * q);
      const double2 bv = *reinterpret_cast<const double2*>(b + 2 * q);
      na[2 * q] = av.x; na[2 * q + 1] = av.y;
      nb[2 * q] = bv.x; nb[2 * q + 1] = bv.y;
    }
  }
  // rows j and j + 1 at x: the values and their ln Q^2 slopes (per unit of v)
  const K g0 = hermite01(c.u, na[0], na[4], na[1], na[5]);
  const K q0 = hermite01(c.u, na[2], na[6], na[3], na[7]);
  const K g1 = hermite01(c.u, nb[0], nb[4], nb[1], nb[5]);
  const K q1 = hermite01(c.u, nb[2], nb[6], nb[3], nb[7]);
  return hermite01(c.v, g0, g1, q0, q1);
}

template <typename K>
__device__ __forceinline__ K pdf_xfx(const PdfView& pv, int flavour, const PdfCell<K>& c) {
  return pdf_xfx_slice(pv, pdf_table<K>(pv) + int64_t(flavour) * pv.slice, c);
}

}  // namespace mf
