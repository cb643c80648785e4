// Tabulated parton densities: loading a set (mf_pdf_create) and the
// interpolation kernel over caller arrays (mf_pdf_eval); the sampling kernels
// interpolate the same tables (mf_pdf.cuh) for the luminosity of lumi = 2.
#include <cmath>
#include <string>
#include <vector>

#include "mf_internal.h"

using namespace mf;
using namespace mf::detail;

struct mf_pdf {
  PdfView view{};
  double* d64 = nullptr;
  float* d32 = nullptr;
  int device = 0, sms = 0;
};

namespace mf {

// Interpolation of one flavour at n points: x and Q^2 in, x f out (FP64 arrays,
// arithmetic in K).  With SMEM the CTA first copies the flavour's node table
// (64 KB in FP32) into shared memory with 16-byte loads, so that the four
// node reads of a point hit shared memory; the points themselves are read and
// written once, coalesced (24 bytes per point of HBM traffic).
template <typename K, bool SMEM>
__global__ void __launch_bounds__(256) k_pdf_eval(PdfView pv, int flavour, int64_t n, const double* __restrict__ x,
                                                  const double* __restrict__ q2, double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const K* fl = pdf_table<K>(pv) + int64_t(flavour) * pv.slice;
  if constexpr (SMEM) {
    const int4* src = reinterpret_cast<const int4*>(fl);
    int4* dst = reinterpret_cast<int4*>(smem_raw);
    const int64_t words = pv.slice * int64_t(sizeof(K)) / 16;
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) dst[w] = __ldg(src + w);
    __syncthreads();
    fl = reinterpret_cast<const K*>(smem_raw);
  }
  // kPts points per thread per pass, their loads issued together (the
  // points are read once: streaming loads and stores), and the next pass's
  // loads issued before this pass's arithmetic, so that each thread keeps
  // HBM requests in flight while it computes
  constexpr int kPts = 4;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int64_t step = kPts * stride;
  double xv[kPts], qv[kPts];
  auto load = [&](int64_t b, double (&xs)[kPts], double (&qs)[kPts]) {
#pragma unroll
    for (int u = 0; u < kPts; ++u) {
      const int64_t e = b + u * stride;
      xs[u] = e < n ? __ldcs(x + e) : 1.0;
      qs[u] = e < n ? __ldcs(q2 + e) : 1.0;
    }
  };
  int64_t e0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  load(e0, xv, qv);
  for (; e0 < n; e0 += step) {
    double xn[kPts], qn[kPts];
    load(e0 + step, xn, qn);
#pragma unroll
    for (int u = 0; u < kPts; ++u) {
      const int64_t e = e0 + u * stride;
      double r;
      if constexpr (sizeof(K) == sizeof(float)) {
        // FP32: the logarithms, the cell and the interpolation in FP32, and
        // no FP64 instruction at all (conversions between FP64 and FP32 issue
        // on the narrow FP64 pipe)
        const PdfCell<float> c = pdf_cell(pv, log_f64_in_f32(xv[u]), log_f64_in_f32(qv[u]));
        r = widen_f32(pdf_xfx_slice(pv, fl, c));
      } else {
        const PdfCell<double> c = pdf_cell(pv, log(xv[u]), log(qv[u]));
        r = pdf_xfx_slice(pv, fl, c);
      }
      if (e < n) __stcs(out + e, r);
    }
#pragma unroll
    for (int u = 0; u < kPts; ++u) {
      xv[u] = xn[u];
      qv[u] = qn[u];
    }
  }
}

namespace detail {
PdfView pdf_view(const mf_pdf* p) { return p->view; }
int pdf_device(const mf_pdf* p) { return p->device; }
}  // namespace detail

}  // namespace mf

namespace {
constexpr size_t kPdfSmemMax = 200 * 1024;

template <typename K, bool SMEM>
cudaError_t pdf_launch(const mf_pdf* p, int flavour, int64_t n, const double* x, const double* q2, double* out,
                       cudaStream_t s) {
  const size_t smem = SMEM ? size_t(p->view.slice) * sizeof(K) : 0;
  cudaError_t e = cudaFuncSetAttribute(k_pdf_eval<K, SMEM>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pdf_eval<K, SMEM>, 256, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int64_t need = (n + 4 * 256 - 1) / (4 * 256);   // four points per thread per pass
  const int64_t cap = int64_t(p->sms) * occ;
  k_pdf_eval<K, SMEM><<<int(need < cap ? need : cap), 256, smem, s>>>(p->view, flavour, n, x, q2, out);
  return cudaGetLastError();
}
}  // namespace

extern "C" {

mf_status mf_pdf_create(int nflav, int nq, int nx, double x_min, double x_max, double q2_min, double q2_max,
                        const double* xf, mf_pdf** out) {
  if (out == nullptr || xf == nullptr) return fail(MF_ERR_ARG, "mf_pdf_create: null argument");
  *out = nullptr;
  if (nflav < 1 || nflav > 64 || nq < 4 || nx < 4 || nq > 4096 || nx > 4096)
    return fail(MF_ERR_ARG, "mf_pdf_create: need 1 <= nflav <= 64 and 4 <= nq, nx <= 4096");
  if (!(x_min > 0 && x_max > x_min && x_max <= 1.0) || !(q2_min > 0 && q2_max > q2_min) || !std::isfinite(q2_max))
    return fail(MF_ERR_ARG, "mf_pdf_create: need 0 < x_min < x_max <= 1 and 0 < q2_min < q2_max");
  const size_t cells = size_t(nflav) * nq * nx;
  for (size_t k = 0; k < cells; ++k)
    if (!std::isfinite(xf[k])) return fail(MF_ERR_ARG, "mf_pdf_create: the table holds a non-finite value");
  mf_pdf* p = new mf_pdf();
  PdfView& v = p->view;
  v.nflav = nflav;
  v.nq = nq;
  v.nx = nx;
  v.t0 = std::log(x_min);
  v.ht = (std::log(x_max) - v.t0) / (nx - 1);
  v.s0 = std::log(q2_min);
  v.hs = (std::log(q2_max) - v.s0) / (nq - 1);
  v.iht = 1.0 / v.ht;
  v.ihs = 1.0 / v.hs;
  v.t0f = float(v.t0);
  v.htf = float(v.ht);
  v.s0f = float(v.s0);
  v.ihtf = float(v.iht);
  v.ihsf = float(v.ihs);
  // a flavour's slice of (f, df, dq, dfq) 4-tuples per node, padded to 64
  // bytes in FP64 and FP32; every slope is the finite difference per unit of
  // the local coordinate: half the difference of the two neighbours inside,
  // the one-sided difference at the first and last node
  v.slice = (int64_t(nq) * nx * 4 + 7) / 8 * 8;
  std::vector<double> t64(size_t(nflav) * v.slice, 0.0);
  std::vector<float> t32(t64.size(), 0.0f);
  auto fd = [](const double* g, int k, int n, int64_t stride) {
    if (k == 0) return g[stride] - g[0];
    if (k == n - 1) return g[(n - 1) * stride] - g[(n - 2) * stride];
    return 0.5 * (g[(k + 1) * stride] - g[(k - 1) * stride]);
  };
  std::vector<double> dq(size_t(nq) * nx);
  for (int f = 0; f < nflav; ++f) {
    const double* tab = xf + size_t(f) * nq * nx;
    for (int l = 0; l < nq; ++l)
      for (int k = 0; k < nx; ++k) dq[size_t(l) * nx + k] = fd(tab + k, l, nq, nx);
    for (int l = 0; l < nq; ++l)
      for (int k = 0; k < nx; ++k) {
        const size_t o = size_t(f) * v.slice + (size_t(l) * nx + k) * 4;
        t64[o] = tab[size_t(l) * nx + k];
        t64[o + 1] = fd(tab + size_t(l) * nx, k, nx, 1);
        t64[o + 2] = dq[size_t(l) * nx + k];
        t64[o + 3] = fd(dq.data() + size_t(l) * nx, k, nx, 1);
        for (int q = 0; q < 4; ++q) t32[o + q] = float(t64[o + q]);
      }
  }
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
  if (e == cudaSuccess) e = cudaMalloc(&p->d64, sizeof(double) * t64.size());
  if (e == cudaSuccess) e = cudaMalloc(&p->d32, sizeof(float) * t32.size());
  if (e == cudaSuccess) e = cudaMemcpy(p->d64, t64.data(), sizeof(double) * t64.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d32, t32.data(), sizeof(float) * t32.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(p->d64);
    cudaFree(p->d32);
    delete p;
    return cuda_fail(e, "mf_pdf_create");
  }
  v.tab64 = p->d64;
  v.tab32 = p->d32;
  *out = p;
  return MF_OK;
}

mf_status mf_pdf_destroy(mf_pdf* p) {
  if (p == nullptr) return MF_OK;
  cudaFree(p->d64);
  cudaFree(p->d32);
  delete p;
  return MF_OK;
}

mf_status mf_pdf_eval(const mf_pdf* p, int precision, int flavour, int64_t n, const double* x, const double* q2,
                      double* xf, void* stream) {
  if (p == nullptr || n < 0) return fail(MF_ERR_ARG, "mf_pdf_eval: bad argument");
  if (flavour < 0 || flavour >= p->view.nflav) return fail(MF_ERR_ARG, "mf_pdf_eval: flavour index out of range");
  if (precision != MF_FP64 && precision != MF_FP32) return fail(MF_ERR_ARG, "mf_pdf_eval: precision MF_FP64 or MF_FP32");
  if (n == 0) return MF_OK;
  if (x == nullptr || q2 == nullptr || xf == nullptr) return fail(MF_ERR_ARG, "mf_pdf_eval: null buffer");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = size_t(p->view.slice) * (precision == MF_FP64 ? sizeof(double) : sizeof(float));
  const bool smem = bytes <= kPdfSmemMax;
  cudaError_t e;
  if (precision == MF_FP64) e = smem ? pdf_launch<double, true>(p, flavour, n, x, q2, xf, s)
                                     : pdf_launch<double, false>(p, flavour, n, x, q2, xf, s);
  else e = smem ? pdf_launch<float, true>(p, flavour, n, x, q2, xf, s)
                : pdf_launch<float, false>(p, flavour, n, x, q2, xf, s);
  if (e != cudaSuccess) return cuda_fail(e, "mf_pdf_eval");
  count_launches(1);
  return MF_OK;
}

}  // extern "C"
