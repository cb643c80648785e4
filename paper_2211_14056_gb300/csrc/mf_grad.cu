// Derivatives of the event weight and of the cross-section estimate with
// respect to m_t, Gamma_t and the Vegas uniforms (arXiv:2211.14056, Sec. 2:
// the custom operator lacks a derivative, "trivial to extend"); the g_s
// derivative is exact from |M|^2 ~ g_s^(2 n_gluons).
//
// Forward mode: the sampling and amplitude code run with dual numbers
// Dual<B, 2> (two tangent directions per pass).  Every wavefunction, current
// and amplitude is recomputed with its tangents inside the pass; nothing is
// stored between passes.  Pass 0 carries (m_t, Gamma_t); further passes carry
// pairs of Vegas uniforms.  Bins and cut decisions are piecewise constant and
// contribute no derivative: d sigma/d theta is the derivative of the estimator
// at fixed uniforms.
#include <cstring>
#include <string>
#include <vector>

#include "mf_internal.h"

namespace mf {

constexpr int kGradTangents = 2;

struct GradArgs {
  SampleParams sp;
  MeParams mp;
  double width;               // Gamma_t
  const double* edges;
  int64_t n;
  uint64_t seed;
  int iter;
  TangentSeeds ts;
  int mt_slot, wt_slot;       // tangent slots of m_t and Gamma_t in the amplitude (-1: none)
  double* partials;           // [gridDim.x][1 + N]: sum w, sum dw/d(slot)
  double* w_out;              // [n] or null: w * w_scale
  double w_scale;
  double* dw_out[kGradTangents];   // [n] each, or null
};

template <int NG, typename B> struct GradMem {
  using T = Dual<B, kGradTangents>;
  static constexpr int kWarpsPerCta = sizeof(B) == sizeof(float) ? 2 : 1;
  __host__ __device__ static size_t al(size_t x) { return (x + 15) & ~size_t(15); }
  __host__ __device__ static size_t warps(int ndim, int nbins) { return al(sizeof(double) * ndim * (nbins + 1)); }
  __host__ __device__ static size_t total(int ndim, int nbins) {
    return warps(ndim, nbins) + WarpMem<NG, T>::bytes * kWarpsPerCta;
  }
};

template <int NG, typename B>
__global__ void __launch_bounds__(32 * GradMem<NG, B>::kWarpsPerCta) k_grad(GradArgs a) {
  using T = Dual<B, kGradTangents>;
  using DD = Dual<double, kGradTangents>;
  constexpr int W = GradMem<NG, B>::kWarpsPerCta;
  constexpr int EPW = Lanes<NG>::EPW, L = Lanes<NG>::L, NEXT = Lanes<NG>::NEXT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* edges = reinterpret_cast<double*>(smem_raw);
  const int ndim = a.sp.ndim, nbins = a.sp.nbins;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int group = lane / L, gl = lane % L;
  unsigned char* wm = smem_raw + GradMem<NG, B>::warps(ndim, nbins) + warp * WarpMem<NG, T>::bytes;
  for (int i = t; i < ndim * (nbins + 1); i += blockDim.x) edges[i] = a.edges[i];
  __syncthreads();
  // amplitude parameters with their tangents
  T mt = T(B(a.mp.mt)), wt = T(B(a.width));
  if (a.mt_slot >= 0) mt.d[a.mt_slot] = B(1);
  if (a.wt_slot >= 0) wt.d[a.wt_slot] = B(1);
  const T mw = mt * wt;
  const unsigned full = 0xffffffffu;
  double s0 = 0.0, s1[kGradTangents] = {0.0, 0.0};
  const int64_t stride = int64_t(gridDim.x) * W * 32;
  for (int64_t base = (int64_t(blockIdx.x) * W + warp) * 32; base < a.n; base += stride) {
    const int64_t e = base + lane;
    const bool valid = e < a.n;
    EventKin<T, DD> k;
    k.pass = 0;
    k.prefactor = DD(0.0);
    if (valid) sample_event<T, DD>(a.sp, edges, a.seed, a.iter, uint64_t(e), k, &a.ts);
    if (!valid) {
      for (int i = 0; i < NEXT; ++i)
        for (int c = 0; c < 4; ++c) k.p[i][c] = T(B(0));
    }
    DD me = DD(0.0);
    unsigned todo = __ballot_sync(full, valid && k.pass);
    while (todo) {
      int src = -1;
      unsigned rest = todo;
#pragma unroll
      for (int g = 0; g < EPW; ++g) {
        const int b = rest ? __ffs(rest) - 1 : -1;
        if (g == group) src = b;
        if (rest) rest &= rest - 1u;
      }
      const int from = src < 0 ? 0 : src;
      T p[NEXT][4];
#pragma unroll
      for (int i = 0; i < NEXT; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) p[i][c] = shfl_any(full, k.p[i][c], from);
      const T v = group_me2<NG, T>(p, wm, group, gl, mt, mw);
#pragma unroll
      for (int g = 0; g < EPW; ++g) {
        const T vg = shfl_any(full, v, g * L);
        const int sg = __shfl_sync(full, src, g * L);
        if (sg == lane) me = DD(vg) * a.mp.norm;
      }
      todo = rest;
    }
    const DD w = valid ? me * k.prefactor : DD(0.0);
    if (valid) {
      if (a.w_out) a.w_out[e] = w.v * a.w_scale;
      for (int s = 0; s < kGradTangents; ++s)
        if (a.dw_out[s]) a.dw_out[s][e] = w.d[s];
    }
    s0 += w.v;
    for (int s = 0; s < kGradTangents; ++s) s1[s] += w.d[s];
  }
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(full, s0, off);
    for (int s = 0; s < kGradTangents; ++s) s1[s] += __shfl_xor_sync(full, s1[s], off);
  }
  __shared__ double acc[1 + kGradTangents];
  if (t <= kGradTangents) acc[t] = 0.0;
  __syncthreads();
  if (lane == 0) {
    atomicAdd(&acc[0], s0);
    for (int s = 0; s < kGradTangents; ++s) atomicAdd(&acc[1 + s], s1[s]);
  }
  __syncthreads();
  if (t <= kGradTangents) a.partials[int64_t(blockIdx.x) * (1 + kGradTangents) + t] = acc[t];
}

template <int NG, typename B>
cudaError_t launch_grad(const GradArgs& a, int sms, int max_grid, int* grid_out, cudaStream_t s) {
  const size_t sm = GradMem<NG, B>::total(a.sp.ndim, a.sp.nbins);
  cudaError_t e = cudaFuncSetAttribute(k_grad<NG, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_grad<NG, B>, 32 * GradMem<NG, B>::kWarpsPerCta, sm);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int64_t per = 32 * GradMem<NG, B>::kWarpsPerCta;
  int64_t grid = (a.n + per - 1) / per;
  if (grid > int64_t(sms) * occ) grid = int64_t(sms) * occ;
  if (grid > max_grid) grid = max_grid;
  k_grad<NG, B><<<int(grid), 32 * GradMem<NG, B>::kWarpsPerCta, sm, s>>>(a);
  *grid_out = int(grid);
  return cudaGetLastError();
}

}  // namespace mf

using namespace mf;
using namespace mf::detail;

extern "C" mf_status mf_grad(mf_process* p, const mf_grid* g, uint64_t seed, int iter, int64_t n, double* sigma,
                             double* dsigma, double* dw_dtheta, double* dw_dy, void* stream) {
  if (p == nullptr || g == nullptr || dsigma == nullptr || sigma == nullptr)
    return fail(MF_ERR_ARG, "mf_grad: null argument");
  if (g->proc != p) return fail(MF_ERR_ARG, "mf_grad: grid belongs to another process");
  if (n < 1) return fail(MF_ERR_ARG, "mf_grad: n must be >= 1");
  if (iter < 0) return fail(MF_ERR_ARG, "mf_grad: iter must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  GradArgs a;
  std::memset(&a, 0, sizeof(a));
  a.sp = p->sp;
  a.sp.nbins = g->nbins;
  a.mp = p->mp;
  a.width = p->width;
  a.edges = g->d_edges;
  a.n = n;
  a.seed = seed;
  a.iter = iter;
  a.partials = g->d_partials;
  const int ndim = g->ndim;
  // the grid's partial-sum scratch holds max_blocks * (2 + ndim * nbins) doubles
  const int64_t slots = int64_t(g->max_blocks) * (2 + int64_t(ndim) * g->nbins);
  const int max_grid = int(slots / (1 + kGradTangents));
  const int power = 2 * p->ng;   // |M|^2 is proportional to g_s^(2 n_gluons)
  double sw = 0.0, dm = 0.0, dg = 0.0;
  // pass 0: (m_t, Gamma_t); passes 1, 2, ...: pairs of Vegas uniforms
  const int passes = 1 + (dw_dy != nullptr ? (ndim + 1) / 2 : 0);
  for (int pass = 0; pass < passes; ++pass) {
    for (int j = 0; j < kMaxDim; ++j) a.ts.y_slot[j] = -1;
    a.ts.mt_slot = -1;
    a.mt_slot = a.wt_slot = -1;
    a.w_out = nullptr;
    a.w_scale = 0.0;
    a.dw_out[0] = a.dw_out[1] = nullptr;
    if (pass == 0) {
      a.ts.mt_slot = 0;
      a.mt_slot = 0;
      a.wt_slot = 1;
      if (dw_dtheta != nullptr) {   // rows g_s, m_t, Gamma_t
        a.w_out = dw_dtheta;
        a.w_scale = power / p->g_s;
        a.dw_out[0] = dw_dtheta + n;
        a.dw_out[1] = dw_dtheta + 2 * n;
      }
    } else {
      const int j0 = 2 * (pass - 1);
      a.ts.y_slot[j0] = 0;
      a.dw_out[0] = dw_dy + int64_t(j0) * n;
      if (j0 + 1 < ndim) {
        a.ts.y_slot[j0 + 1] = 1;
        a.dw_out[1] = dw_dy + int64_t(j0 + 1) * n;
      }
    }
    int grid = 0;
    cudaError_t e;
    const bool fp64 = p->precision == MF_FP64;
    switch (p->ng) {
      case 2: e = fp64 ? launch_grad<2, double>(a, p->sms, max_grid, &grid, s) : launch_grad<2, float>(a, p->sms, max_grid, &grid, s); break;
      case 3: e = fp64 ? launch_grad<3, double>(a, p->sms, max_grid, &grid, s) : launch_grad<3, float>(a, p->sms, max_grid, &grid, s); break;
      default: e = fp64 ? launch_grad<4, double>(a, p->sms, max_grid, &grid, s) : launch_grad<4, float>(a, p->sms, max_grid, &grid, s); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "mf_grad (kernel)");
    count_launches(1);
    if (pass == 0) {
      std::vector<double> host(size_t(grid) * (1 + kGradTangents));
      MF_CUDA(cudaMemcpyAsync(host.data(), g->d_partials, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, s),
              "mf_grad (copy)");
      MF_CUDA(cudaStreamSynchronize(s), "mf_grad (sync)");
      for (int b = 0; b < grid; ++b) {
        sw += host[size_t(b) * 3 + 0];
        dm += host[size_t(b) * 3 + 1];
        dg += host[size_t(b) * 3 + 2];
      }
    }
  }
  MF_CUDA(cudaStreamSynchronize(s), "mf_grad (sync)");
  const double dn = double(n);
  *sigma = sw / dn;
  dsigma[0] = power * (*sigma) / p->g_s;
  dsigma[1] = dm / dn;
  dsigma[2] = dg / dn;
  return MF_OK;
}
