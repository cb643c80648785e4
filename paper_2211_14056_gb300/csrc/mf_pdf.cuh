// Parton densities from a table: log-bicubic Hermite interpolation of
// x f(x, Q^2) (arXiv:2211.14056 Sec. 1: the integrand's densities come from
// PDFFlow, the GPU interpolation of tabulated LHAPDF sets).
//
// A set is stored per flavour as nq rows (ln Q^2 nodes) of nx nodes (ln x),
// uniform in both logarithms; every node holds the pair (x f, d(x f)/d ln x),
// the slope taken once when the table is loaded from the finite differences of
// the node values (mean of the two neighbouring quotients, one-sided at the
// first and last node).  A query (x, Q^2) is clamped to the table's range and
// located in cell (i, j); each of the rows j-1 .. j+2 that exists is a cubic
// Hermite polynomial in ln x on [t_i, t_i+1]; their values then give the ln Q^2
// slopes at s_j and s_j+1 by the same finite differences, and a cubic Hermite
// step in ln Q^2 finishes.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mf {

constexpr int kMaxPdfPairs = 8;

// Device view of a loaded set: node tables in FP64 and FP32, flavour-major,
// each flavour's slice padded to `slice` elements (pairs counted as two).
struct PdfView {
  const double* tab64;
  const float* tab32;
  int nflav, nq, nx;
  int64_t slice;            // elements per flavour (>= nq * nx * 2)
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

template <typename K> __device__ __forceinline__ K pdf_ht(const PdfView& pv);
template <> __device__ __forceinline__ double pdf_ht<double>(const PdfView& pv) { return pv.ht; }
template <> __device__ __forceinline__ float pdf_ht<float>(const PdfView& pv) { return pv.htf; }

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
// error below 2^-23), ln x = e ln 2 + ln m with ln 2 in two parts.  x <= 0
// or subnormal gives a large negative value (the callers clamp to the table).
__device__ __forceinline__ float log_f64_in_f32(double x) {
  const long long b = __double_as_longlong(x);
  const int e = int((b >> 52) & 0x7ff) - 1023;
  const float m = __int_as_float(0x3f800000 | int((b >> 29) & 0x7fffff));
  const float fe = float(e);
  return fmaf(fe, 1.428606765330187e-06f, fmaf(fe, 0.693145751953125f, logf(m)));
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

// one row (ln Q^2 node l) of flavour slice `fl` at the cell's x
template <typename K>
__device__ __forceinline__ K pdf_row(const K* fl, int nx, int l, int i, K u, K ht) {
  const K* r = fl + (int64_t(l) * nx + i) * 2;
  return hermite01(u, r[0], r[2], ht * r[1], ht * r[3]);
}

// x f(x, Q^2) of the flavour whose slice starts at `fl`
template <typename K>
__device__ __forceinline__ K pdf_xfx_slice(const PdfView& pv, const K* fl, const PdfCell<K>& c) {
  const int nq = pv.nq, j = c.j;
  const K ht = pdf_ht<K>(pv);
  const K g0 = pdf_row(fl, pv.nx, j, c.i, c.u, ht);
  const K g1 = pdf_row(fl, pv.nx, j + 1, c.i, c.u, ht);
  // slopes per ln Q^2 step at s_j and s_j+1 (times the step: per unit of v)
  K d0 = g1 - g0, d1 = g1 - g0;
  if (j > 0) d0 = K(0.5) * (g1 - pdf_row(fl, pv.nx, j - 1, c.i, c.u, ht));
  if (j + 2 <= nq - 1) d1 = K(0.5) * (pdf_row(fl, pv.nx, j + 2, c.i, c.u, ht) - g0);
  return hermite01(c.v, g0, g1, d0, d1);
}

template <typename K>
__device__ __forceinline__ K pdf_xfx(const PdfView& pv, int flavour, const PdfCell<K>& c) {
  return pdf_xfx_slice(pv, pdf_table<K>(pv) + int64_t(flavour) * pv.slice, c);
}

}  // namespace mf
