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
__device__ __forceinline__ void pdf_locate(K z, double c0, double ih, int n, int& cell, K& loc) {
  K r = (z - K(c0)) * K(ih);
  r = r < K(0) ? K(0) : (r > K(n - 1) ? K(n - 1) : r);
  int k = int(r);
  k = k > n - 2 ? n - 2 : k;
  cell = k;
  loc = r - K(k);
}

template <typename K>
__device__ __forceinline__ PdfCell<K> pdf_cell(const PdfView& pv, K lnx, K lnq2) {
  PdfCell<K> c;
  pdf_locate(lnx, pv.t0, pv.iht, pv.nx, c.i, c.u);
  pdf_locate(lnq2, pv.s0, pv.ihs, pv.nq, c.j, c.v);
  return c;
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
  const K ht = K(pv.ht);
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
