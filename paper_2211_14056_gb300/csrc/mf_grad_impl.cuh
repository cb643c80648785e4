// Kernels and host drivers of the derivative pass (included by the
// mf_grad_ng*.cu translation units, each instantiating one gluon count and
// mode): the dual sampling kernel, the forward-mode amplitude kernel, the
// adjoint kernel's launch (mf_adjoint.cuh), the sampler-only tangent passes.
#pragma once
#include <cstring>
#include <string>
#include <vector>

#include "mf_adjoint.cuh"
#include "mf_grad.h"

namespace mf {

// Dual per-event records of one chunk of C events (the derivative pass's
// counterpart of RecordView): momenta and sqrt(s_hat) with their tangents in
// the amplitude's type, the weight prefactor with its tangents in FP64, and
// the list of events that passed.
template <typename B> struct GradRec {
  using T = Dual<B, kGradTangents>;
  using DD = Dual<double, kGradTangents>;
  T* mom;                     // [n_final * 4][C]
  T* rs;                      // [C]
  DD* pref;                   // [C]
  int* list;                  // [C]
  unsigned* count;            // [2]
  int64_t C;
  __host__ __device__ static size_t al(size_t x) { return (x + 255) & ~size_t(255); }
  __host__ __device__ static size_t bytes(int n_final, int64_t C) {
    size_t o = al(sizeof(T) * (size_t(n_final) * 4 + 1) * C);
    o = al(o + sizeof(DD) * C);
    o = al(o + sizeof(int) * C);
    return o + 2 * sizeof(unsigned);
  }
  __host__ __device__ static GradRec carve(void* base, int n_final, int64_t C) {
    GradRec r;
    unsigned char* p = static_cast<unsigned char*>(base);
    r.C = C;
    r.mom = reinterpret_cast<T*>(p);
    r.rs = r.mom + size_t(n_final) * 4 * C;
    size_t o = al(sizeof(T) * (size_t(n_final) * 4 + 1) * C);
    r.pref = reinterpret_cast<DD*>(p + o);
    o = al(o + sizeof(DD) * C);
    r.list = reinterpret_cast<int*>(p + o);
    o = al(o + sizeof(int) * C);
    r.count = reinterpret_cast<unsigned*>(p + o);
    return r;
  }
};

// Dual sampling: one thread per event; events that fail the cuts get zero
// outputs here, the others are listed for the amplitude kernel.
template <typename B>
__global__ void __launch_bounds__(kThreads) k_grad_sample(GradArgs a, GradRec<B> rec, int64_t out_off) {
  using T = Dual<B, kGradTangents>;
  using DD = Dual<double, kGradTangents>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* edges = reinterpret_cast<double*>(smem_raw);
  for (int i = threadIdx.x; i < a.sp.ndim * (a.sp.nbins + 1); i += blockDim.x) edges[i] = a.edges[i];
  __syncthreads();
  const int nf = a.sp.n_final;
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < a.n; base += stride) {
    const int64_t e = base + threadIdx.x;
    int pass = 0;
    if (e < a.n) {
      EventKin<T, DD> k;
      sample_event<T, DD>(a.sp, edges, a.seed, a.iter, uint64_t(a.first + e), k, &a.ts);
#pragma unroll
      for (int i = 0; i < kMaxExt - 2; ++i)
        if (i < nf)
#pragma unroll
          for (int c = 0; c < 4; ++c) rec.mom[int64_t(i * 4 + c) * rec.C + e] = k.p[2 + i][c];
      rec.rs[e] = k.p[0][0] + k.p[1][0];
      rec.pref[e] = k.prefactor;
      pass = k.pass;
      if (!pass) {
        const int64_t o = out_off + e;
        if (a.w_out) a.w_out[o] = 0.0;
        for (int s = 0; s < kGradTangents; ++s)
          if (a.dw_out[s]) a.dw_out[s][o] = 0.0;
        if (a.dw_mt) a.dw_mt[o] = 0.0;
        if (a.dw_wt) a.dw_wt[o] = 0.0;
      }
    }
    const unsigned bal = __ballot_sync(full, pass);
    unsigned pos = 0;
    if (lane == 0 && bal) pos = atomicAdd(&rec.count[0], unsigned(__popc(bal)));
    pos = __shfl_sync(full, pos, 0);
    if (pass) rec.list[pos + __popc(bal & ((1u << lane) - 1u))] = int(e);
  }
}

// Dual |M|^2 of the listed events (one lane group per event, as in the plain
// list-based kernel), the weight and its tangents, per-CTA sums.
template <int NG, typename B>
__global__ void __launch_bounds__(32) k_grad_me(GradArgs a, GradRec<B> rec, int64_t out_off) {
  using T = Dual<B, kGradTangents>;
  using DD = Dual<double, kGradTangents>;
  constexpr int EPW = Lanes<NG>::EPW, L = Lanes<NG>::L, NEXT = Lanes<NG>::NEXT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* wm = smem_raw;
  const int lane = threadIdx.x & 31, group = lane / L, gl = lane % L;
  T mt = T(B(a.mp.mt)), wt = T(B(a.width));
  if (a.mt_slot >= 0) mt.d[a.mt_slot] = B(1);
  if (a.wt_slot >= 0) wt.d[a.wt_slot] = B(1);
  const T mw = mt * wt;
  const unsigned full = 0xffffffffu;
  const int64_t npass = rec.count[0];
  double s0 = 0.0, s1[kGradTangents] = {0.0, 0.0};
  for (int64_t base = int64_t(blockIdx.x) * EPW; base < npass; base += int64_t(gridDim.x) * EPW) {
    const int64_t k = base + group;
    const bool ok = k < npass;
    const int64_t e = rec.list[ok ? k : base];
    T p[NEXT][4];
    const T rs = rec.rs[e];
    const T h = rs * B(0.5);
    p[0][0] = h; p[0][1] = T(B(0)); p[0][2] = T(B(0)); p[0][3] = h;
    p[1][0] = h; p[1][1] = T(B(0)); p[1][2] = T(B(0)); p[1][3] = -h;
#pragma unroll
    for (int i = 0; i < NG; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) p[2 + i][c] = rec.mom[int64_t(i * 4 + c) * rec.C + e];
    const T v = group_me2<NG, T>(p, wm, group, gl, mt, mw);
    if (ok && gl == 0) {
      const DD w = DD(v) * a.mp.norm * rec.pref[e];
      const int64_t o = out_off + e;
      if (a.w_out) a.w_out[o] = w.v * a.w_scale;
      for (int s = 0; s < kGradTangents; ++s)
        if (a.dw_out[s]) a.dw_out[s][o] = w.d[s];
      s0 += w.v;
      for (int s = 0; s < kGradTangents; ++s) s1[s] += w.d[s];
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(full, s0, off);
    for (int s = 0; s < kGradTangents; ++s) s1[s] += __shfl_xor_sync(full, s1[s], off);
  }
  if (lane <= kGradTangents) {
    const double v = lane == 0 ? s0 : s1[lane - 1];
    double* dst = a.partials + int64_t(blockIdx.x) * (1 + kGradTangents) + lane;
    *dst = (a.accumulate ? *dst : 0.0) + v;
  }
}

// per-event adjoint record: |M|^2, d|M|^2/dp[2 + i][c] (i < 4), d|M|^2/d sqrt(s_hat)
constexpr int kAdjStride = 1 + 16 + 1;

// Adjoint |M|^2 of the listed events (one lane group per event), contracted
// with the records' two tangents; per-CTA sums of w, dw/dm_t, dw/dGamma_t.
template <int NG, typename B>
__global__ void __launch_bounds__(32, 8) k_adj_me(GradArgs a, GradRec<B> rec, int64_t out_off) {
  using TD = Dual<B, kGradTangents>;
  using DD = Dual<double, kGradTangents>;
  constexpr int EPW = Lanes<NG>::EPW, L = Lanes<NG>::L, NEXT = Lanes<NG>::NEXT;
  constexpr int NR = AdjRows<NG>::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, group = lane / L, gl = lane % L;
  const B mt = B(a.mp.mt), wt = B(a.width), mw = mt * wt;
  const unsigned full = 0xffffffffu;
  const int64_t npass = rec.count[0];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int64_t base = int64_t(blockIdx.x) * EPW; base < npass; base += int64_t(gridDim.x) * EPW) {
    const int64_t k = base + group;
    const bool ok = k < npass;
    const int64_t e = rec.list[ok ? k : base];
    B p[NEXT][4];
    const TD rs = rec.rs[e];
    const B h = B(0.5) * rs.v;
    p[0][0] = h; p[0][1] = B(0); p[0][2] = B(0); p[0][3] = h;
    p[1][0] = h; p[1][1] = B(0); p[1][2] = B(0); p[1][3] = -h;
#pragma unroll
    for (int i = 0; i < NG; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) p[2 + i][c] = rec.mom[int64_t(i * 4 + c) * rec.C + e].v;
    B ad[NR];
    const B me = adj_group_me2<NG, B>(p, smem_raw, group, gl, mt, mw, B(a.mp.norm), ad);
    if (ok && gl == 0) {
      const DD pref = rec.pref[e];
      const double rsb = 0.5 * (double(ad[0]) + double(ad[3]) + double(ad[4]) - double(ad[7]));
      const double mb = double(ad[AdjRows<NG>::MB]) + double(wt) * double(ad[AdjRows<NG>::MWB]);
      const double wb = double(mt) * double(ad[AdjRows<NG>::MWB]);
      const double w = double(me) * pref.v;
      double dme[kGradTangents];
#pragma unroll
      for (int t = 0; t < kGradTangents; ++t) {
        double x = rsb * double(rs.d[t]);
#pragma unroll
        for (int i = 0; i < NG; ++i)
#pragma unroll
          for (int c = 0; c < 4; ++c) x += double(ad[(2 + i) * 4 + c]) * double(rec.mom[int64_t(i * 4 + c) * rec.C + e].d[t]);
        if (t == a.mt_tan) x += mb;
        dme[t] = x * pref.v + double(me) * pref.d[t];
      }
      const int64_t o = out_off + e;
      if (a.w_out) a.w_out[o] = w * a.w_scale;
      for (int t = 0; t < kGradTangents; ++t)
        if (a.dw_out[t]) a.dw_out[t][o] = dme[t];
      if (a.dw_mt) a.dw_mt[o] = a.mt_tan >= 0 ? dme[a.mt_tan] : 0.0;
      if (a.dw_wt) a.dw_wt[o] = wb * pref.v;
      double* r = a.adj + e * kAdjStride;
      r[0] = double(me);
      for (int i = 0; i < NG; ++i)
        for (int c = 0; c < 4; ++c) r[1 + i * 4 + c] = double(ad[(2 + i) * 4 + c]);
      r[kAdjStride - 1] = rsb;
      s0 += w;
      s1 += a.mt_tan >= 0 ? dme[a.mt_tan] : 0.0;
      s2 += wb * pref.v;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(full, s0, off);
    s1 += __shfl_xor_sync(full, s1, off);
    s2 += __shfl_xor_sync(full, s2, off);
  }
  if (lane < 3) {
    const double v = lane == 0 ? s0 : lane == 1 ? s1 : s2;
    double* dst = a.partials + int64_t(blockIdx.x) * 3 + lane;
    *dst = (a.accumulate ? *dst : 0.0) + v;
  }
}

// A tangent pass of the sampler alone: two more uniforms per pass, contracted
// with the stored per-event adjoint (one thread per event).
template <typename B>
__global__ void __launch_bounds__(kThreads) k_grad_tangent(GradArgs a, int64_t out_off) {
  using TD = Dual<B, kGradTangents>;
  using DD = Dual<double, kGradTangents>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* edges = reinterpret_cast<double*>(smem_raw);
  for (int i = threadIdx.x; i < a.sp.ndim * (a.sp.nbins + 1); i += blockDim.x) edges[i] = a.edges[i];
  __syncthreads();
  const int nf = a.sp.n_final;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < a.n; e += int64_t(gridDim.x) * blockDim.x) {
    EventKin<TD, DD> k;
    sample_event<TD, DD>(a.sp, edges, a.seed, a.iter, uint64_t(a.first + e), k, &a.ts);
    const double* r = a.adj + e * kAdjStride;
    const int64_t o = out_off + e;
#pragma unroll
    for (int t = 0; t < kGradTangents; ++t) {
      if (!a.dw_out[t]) continue;
      double x = 0.0;
      if (k.pass) {
        x = r[kAdjStride - 1] * double((k.p[0][0] + k.p[1][0]).d[t]);
#pragma unroll
        for (int i = 0; i < kMaxExt - 2; ++i)
          if (i < nf)
#pragma unroll
            for (int c = 0; c < 4; ++c) x += r[1 + i * 4 + c] * double(k.p[2 + i][c].d[t]);
        x = x * k.prefactor.v + r[0] * k.prefactor.d[t];
      }
      a.dw_out[t][o] = x;
    }
  }
}

template <int NG, typename B>
cudaError_t adj_me_config(int* occ, size_t* smem) {
  *smem = AdjMem<NG, B>::bytes;
  cudaError_t e = cudaFuncSetAttribute(k_adj_me<NG, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_adj_me<NG, B>, 32, *smem);
}

template <int NG, typename B>
cudaError_t grad_me_config(int* occ, size_t* smem) {
  using T = Dual<B, kGradTangents>;
  *smem = WarpMem<NG, T>::bytes;
  cudaError_t e = cudaFuncSetAttribute(k_grad_me<NG, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_grad_me<NG, B>, 32, *smem);
}

// one chunk: sampling, then the amplitude kernel on a fixed persistent grid
template <int NG, typename B>
cudaError_t launch_grad_chunk(const GradArgs& a, void* rec_base, int64_t C, int me_grid, int64_t out_off,
                              cudaStream_t s) {
  GradRec<B> rec = GradRec<B>::carve(rec_base, a.sp.n_final, C);
  cudaError_t e = cudaMemsetAsync(rec.count, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t need = (a.n + kThreads - 1) / kThreads;
  const int sgrid = int(need < int64_t(sms) * 8 ? need : int64_t(sms) * 8);
  const size_t esm = sizeof(double) * a.sp.ndim * (a.sp.nbins + 1);
  k_grad_sample<B><<<sgrid, kThreads, esm, s>>>(a, rec, out_off);
  using T = Dual<B, kGradTangents>;
  k_grad_me<NG, B><<<me_grid, 32, WarpMem<NG, T>::bytes, s>>>(a, rec, out_off);
  return cudaGetLastError();
}

namespace gradimpl {

using namespace mf::detail;


template <int NG, typename B>
mf_status grad_forward(mf_process* p, const mf_grid* g, GradArgs& a, int64_t n, double* dw_dtheta, double* dw_dy,
                      int power, double* sums, cudaStream_t s) {
  const int ndim = g->ndim;
  int occ = 0;
  size_t msm = 0;
  MF_CUDA((grad_me_config<NG, B>(&occ, &msm)), "mf_grad (configuration)");
  if (occ < 1) return fail(MF_ERR_CUDA, "mf_grad: amplitude kernel does not fit on an SM");
  // the grid's partial-sum scratch holds max_blocks * (2 + ndim * nbins) doubles
  const int64_t slots = int64_t(g->max_blocks) * (2 + int64_t(ndim) * g->nbins);
  int me_grid = p->sms * occ;
  if (int64_t(me_grid) * (1 + kGradTangents) > slots) me_grid = int(slots / (1 + kGradTangents));
  const int64_t C = n < (int64_t(1) << 18) ? n : (int64_t(1) << 18);
  void* rec = nullptr;
  MF_CUDA(cudaMallocAsync(&rec, GradRec<B>::bytes(p->sp.n_final, C), s), "mf_grad (records)");
  const int passes = 1 + (dw_dy != nullptr ? (ndim + 1) / 2 : 0);
  mf_status st = MF_OK;
  for (int pass = 0; pass < passes && st == MF_OK; ++pass) {
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
    for (int64_t done = 0; done < n; done += C) {
      const int64_t m = n - done < C ? n - done : C;
      a.first = done;
      a.n = m;
      a.accumulate = done > 0;
      cudaError_t e = launch_grad_chunk<NG, B>(a, rec, C, me_grid, done, s);
      if (e != cudaSuccess) { st = cuda_fail(e, "mf_grad (kernels)"); break; }
      count_launches(2);
    }
    if (st == MF_OK && pass == 0) {
      std::vector<double> host(size_t(me_grid) * (1 + kGradTangents));
      cudaError_t e = cudaMemcpyAsync(host.data(), g->d_partials, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) { st = cuda_fail(e, "mf_grad (sums)"); break; }
      for (int b = 0; b < me_grid; ++b)
        for (int k = 0; k <= kGradTangents; ++k) sums[k] += host[size_t(b) * (1 + kGradTangents) + k];
    }
  }
  cudaFreeAsync(rec, s);
  return st;
}

// reverse mode: per chunk, pass 0 (dual sampling with m_t and y_0, the
// adjoint kernel), then the sampler-only tangent passes for y_1 ..
template <int NG, typename B>
mf_status grad_adjoint(mf_process* p, const mf_grid* g, GradArgs& a, int64_t n, double* dw_dtheta, double* dw_dy,
                       int power, double* sums, cudaStream_t s) {
  const int ndim = g->ndim;
  int occ = 0;
  size_t msm = 0;
  MF_CUDA((adj_me_config<NG, B>(&occ, &msm)), "mf_grad (configuration)");
  if (occ < 1) return fail(MF_ERR_CUDA, "mf_grad: adjoint kernel does not fit on an SM");
  const int64_t slots = int64_t(g->max_blocks) * (2 + int64_t(ndim) * g->nbins);
  int me_grid = p->sms * occ;
  if (int64_t(me_grid) * 3 > slots) me_grid = int(slots / 3);
  const int64_t C = n < (int64_t(1) << 18) ? n : (int64_t(1) << 18);
  void* rec = nullptr;
  double* adj = nullptr;
  MF_CUDA(cudaMallocAsync(&rec, GradRec<B>::bytes(p->sp.n_final, C), s), "mf_grad (records)");
  cudaError_t e0 = cudaMallocAsync(reinterpret_cast<void**>(&adj), sizeof(double) * kAdjStride * C, s);
  if (e0 != cudaSuccess) {
    cudaFreeAsync(rec, s);
    return cuda_fail(e0, "mf_grad (adjoint records)");
  }
  a.adj = adj;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t esm = sizeof(double) * a.sp.ndim * (a.sp.nbins + 1);
  mf_status st = MF_OK;
  for (int64_t done = 0; done < n && st == MF_OK; done += C) {
    const int64_t m = n - done < C ? n - done : C;
    a.first = done;
    a.n = m;
    const int64_t need = (m + kThreads - 1) / kThreads;
    const int sgrid = int(need < int64_t(sms) * 8 ? need : int64_t(sms) * 8);
    // pass 0
    for (int j = 0; j < kMaxDim; ++j) a.ts.y_slot[j] = -1;
    a.ts.mt_slot = 0;
    a.mt_tan = 0;
    a.accumulate = done > 0;
    a.w_out = dw_dtheta;
    a.w_scale = power / p->g_s;
    a.dw_mt = dw_dtheta ? dw_dtheta + n : nullptr;
    a.dw_wt = dw_dtheta ? dw_dtheta + 2 * n : nullptr;
    a.dw_out[0] = nullptr;
    a.dw_out[1] = nullptr;
    if (dw_dy != nullptr) {
      a.ts.y_slot[0] = 1;
      a.dw_out[1] = dw_dy;
    }
    GradRec<B> gr = GradRec<B>::carve(rec, a.sp.n_final, C);
    cudaError_t e = cudaMemsetAsync(gr.count, 0, 2 * sizeof(unsigned), s);
    if (e == cudaSuccess) {
      k_grad_sample<B><<<sgrid, kThreads, esm, s>>>(a, gr, done);
      k_adj_me<NG, B><<<me_grid, 32, msm, s>>>(a, gr, done);
      e = cudaGetLastError();
      count_launches(2);
    }
    if (e != cudaSuccess) { st = cuda_fail(e, "mf_grad (kernels)"); break; }
    // tangent passes of the remaining uniforms
    if (dw_dy != nullptr) {
      a.ts.mt_slot = -1;
      a.mt_tan = -1;
      for (int j0 = 1; j0 < ndim; j0 += 2) {
        for (int j = 0; j < kMaxDim; ++j) a.ts.y_slot[j] = -1;
        a.ts.y_slot[j0] = 0;
        a.dw_out[0] = dw_dy + int64_t(j0) * n;
        a.dw_out[1] = nullptr;
        if (j0 + 1 < ndim) {
          a.ts.y_slot[j0 + 1] = 1;
          a.dw_out[1] = dw_dy + int64_t(j0 + 1) * n;
        }
        k_grad_tangent<B><<<sgrid, kThreads, esm, s>>>(a, done);
        e = cudaGetLastError();
        count_launches(1);
        if (e != cudaSuccess) { st = cuda_fail(e, "mf_grad (tangent pass)"); break; }
      }
    }
  }
  if (st == MF_OK) {
    std::vector<double> host(size_t(me_grid) * 3);
    cudaError_t e = cudaMemcpyAsync(host.data(), g->d_partials, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "mf_grad (sums)");
    else
      for (int b = 0; b < me_grid; ++b)
        for (int k = 0; k < 3; ++k) sums[k] += host[size_t(b) * 3 + k];
  }
  cudaFreeAsync(adj, s);
  cudaFreeAsync(rec, s);
  return st;
}

}  // namespace gradimpl
}  // namespace mf
