// Precision- and process-independent kernels: per-event sampling, and the
// deterministic reduction of per-CTA Vegas partials followed by the grid
// refinement (Lepage 1980; arXiv:2211.14056 Sec. 1 names Vegas as its integrator).
#include "mf_kernels.cuh"

namespace mf {

__global__ void __launch_bounds__(kThreads) k_sample(SampleParams sp, const double* __restrict__ edges_g, int64_t n,
                                                     uint64_t seed, int iter, double* __restrict__ mom,
                                                     double* __restrict__ wps, uint8_t* __restrict__ bins) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* edges = reinterpret_cast<double*>(smem_raw);
  for (int i = threadIdx.x; i < sp.ndim * (sp.nbins + 1); i += blockDim.x) edges[i] = edges_g[i];
  __syncthreads();
  const int next = sp.n_final + 2;
  for (int64_t ev = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; ev < n; ev += int64_t(gridDim.x) * blockDim.x) {
    EventKin<double> k;
    sample_event(sp, edges, seed, iter, uint64_t(ev), k);
    if (mom != nullptr)
#pragma unroll
      for (int i = 0; i < kMaxExt; ++i)
        if (i < next)
#pragma unroll
          for (int c = 0; c < 4; ++c) mom[int64_t(i * 4 + c) * n + ev] = k.p[i][c];
    if (wps != nullptr) wps[ev] = k.prefactor;
    if (bins != nullptr)
#pragma unroll
      for (int j = 0; j < kMaxDim; ++j)
        if (j < sp.ndim) bins[int64_t(j) * n + ev] = k.bins[j];
  }
}

// The uniforms alone: y[j][e] of global event first_event + e (the same
// Philox stream every sampling kernel draws from), coalesced FP64 stores.
__global__ void __launch_bounds__(kThreads) k_uniforms(uint64_t seed, int iter, int64_t first_event, int64_t n,
                                                       int ndim, double* __restrict__ y) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    double u[kMaxDim];
    draw_uniforms(seed, iter, uint64_t(first_event + e), ndim, u);
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j)
      if (j < ndim) y[int64_t(j) * n + e] = u[j];
  }
}

cudaError_t launch_uniforms(uint64_t seed, int iter, int64_t first_event, int64_t n, int ndim, double* y,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t need = (n + kThreads - 1) / kThreads;
  const int grid = int(need < int64_t(sms) * 16 ? need : int64_t(sms) * 16);
  k_uniforms<<<grid, kThreads, 0, s>>>(seed, iter, first_event, n, ndim, y);
  return cudaGetLastError();
}

// Hit-or-miss unweighting of one chunk of evaluated events: event e (global
// index first_event + e) with weight w[e] > 0 is kept if r w_max < w[e], r from
// the unweighting stream; a kept event is written at the next free slot (warp-
// aggregated atomics, so the order of the kept events is not fixed, their set
// is): its global index, its weight max(1, w / w_max) and its momenta (beams
// from sqrt(s_hat), final particles from the record), FP64 SoA [n_final + 2][4][cap].
// counts[0] = events kept (may exceed cap: only the first cap are written),
// counts[1] = overweight events kept.
template <typename K>
__global__ void __launch_bounds__(kThreads) k_unweight(RecordView<K> rec, const double* __restrict__ w, int64_t n,
                                                       int n_final, uint64_t seed, int iter, int64_t first_event,
                                                       double w_max, int64_t cap, double* __restrict__ mom_out,
                                                       double* __restrict__ weight_out,
                                                       int64_t* __restrict__ event_out,
                                                       unsigned long long* __restrict__ counts) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < n; base += stride) {
    const int64_t e = base + threadIdx.x;
    double we = 0.0;
    bool keep = false;
    if (e < n) {
      we = w[e];
      if (we > 0.0) keep = __dmul_rn(unweight_uniform(seed, iter, uint64_t(first_event + e)), w_max) < we;
    }
    const unsigned bal = __ballot_sync(full, keep);
    const unsigned over = __ballot_sync(full, keep && we > w_max);
    unsigned long long slot0 = 0;
    if (lane == 0 && bal) {
      slot0 = atomicAdd(&counts[0], (unsigned long long)__popc(bal));
      if (over) atomicAdd(&counts[1], (unsigned long long)__popc(over));
    }
    slot0 = __shfl_sync(full, slot0, 0);
    const int64_t slot = int64_t(slot0) + __popc(bal & ((1u << lane) - 1u));
    if (keep && slot < cap) {
      event_out[slot] = first_event + e;
      weight_out[slot] = we > w_max ? we / w_max : 1.0;
      const double h = 0.5 * double(rec.rs[e]);
      const double beams[2][4] = {{h, 0.0, 0.0, h}, {h, 0.0, 0.0, -h}};
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) mom_out[int64_t(i * 4 + c) * cap + slot] = beams[i][c];
#pragma unroll
      for (int i = 0; i < kMaxExt - 2; ++i)
        if (i < n_final)
#pragma unroll
          for (int c = 0; c < 4; ++c)
            mom_out[int64_t((2 + i) * 4 + c) * cap + slot] = double(rec.mom[int64_t(i * 4 + c) * rec.C + e]);
    }
  }
}

cudaError_t launch_unweight(int precision, void* rec_base, int n_final, int ndim, int64_t C, const double* w,
                            int64_t n, uint64_t seed, int iter, int64_t first_event, double w_max, int64_t cap,
                            double* mom_out, double* weight_out, int64_t* event_out, unsigned long long* counts,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t need = (n + kThreads - 1) / kThreads;
  const int grid = int(need < int64_t(sms) * 16 ? need : int64_t(sms) * 16);
  if (precision == 0)
    k_unweight<double><<<grid, kThreads, 0, s>>>(RecordView<double>::carve(rec_base, n_final, ndim, C), w, n, n_final,
                                                 seed, iter, first_event, w_max, cap, mom_out, weight_out, event_out,
                                                 counts);
  else
    k_unweight<float><<<grid, kThreads, 0, s>>>(RecordView<float>::carve(rec_base, n_final, ndim, C), w, n, n_final,
                                                seed, iter, first_event, w_max, cap, mom_out, weight_out, event_out,
                                                counts);
  return cudaGetLastError();
}

size_t record_bytes(int precision, int n_final, int ndim, int64_t C) {
  return precision == 0 ? RecordView<double>::bytes(n_final, ndim, C) : RecordView<float>::bytes(n_final, ndim, C);
}

cudaError_t launch_sample(const SampleParams& sp, const double* edges, int64_t n, uint64_t seed, int iter,
                          double* mom, double* wps, uint8_t* bins, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t need = (n + kThreads - 1) / kThreads;
  const int grid = int(need < int64_t(sms) * 16 ? need : int64_t(sms) * 16);
  const size_t smem = sizeof(double) * sp.ndim * (sp.nbins + 1);
  k_sample<<<grid, kThreads, smem, s>>>(sp, edges, n, seed, iter, mom, wps, bins);
  return cudaGetLastError();
}

// Lepage's refinement of one dimension by one warp: smooth the per-bin sums
// of w^2 (neighbour average, halves at the ends), normalise, damp with
// ((1 - d)/ln(1/d))^alpha (0 -> 0, 1 -> 1), then place the new edges at equal
// shares of the damped weights, linear inside the old bins.  Lane l holds
// bins l and l + 32 (nb <= 64); the normalising sum is a shuffle reduction,
// the cumulative weights an in-order prefix scan, and each new edge finds its
// old bin by binary search (the largest j < nb with cum[j] <= target).
// cum, old, rw: this dimension's shared scratch (nb + 1, nb + 1, nb doubles).
__device__ void refine_dim_warp(double* e, const double* d, int nb, double alpha, double* cum, double* old,
                                double* rw) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  bool any = false;
  double ds[2], r[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int b = lane + 32 * q;
    ds[q] = 0.0;
    if (b < nb) {
      any |= d[b] > 0.0;
      if (b == 0) ds[q] = (d[0] + d[1]) / 2.0;
      else if (b == nb - 1) ds[q] = (d[nb - 2] + d[nb - 1]) / 2.0;
      else ds[q] = (d[b - 1] + d[b] + d[b + 1]) / 3.0;
    }
  }
  if (!__any_sync(full, any)) return;
  double sum = ds[0] + ds[1];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(full, sum, off);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double dn = ds[q] / sum;
    r[q] = (dn > 0.0 && dn < 1.0) ? pow((1.0 - dn) / log(1.0 / dn), alpha) : (dn >= 1.0 ? 1.0 : 0.0);
  }
  // inclusive prefix sums in bin order: bins 0..31, then 32..63 offset by the first half
  double base = 0.0;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    double x = r[q];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const double y = __shfl_up_sync(full, x, off);
      if (lane >= off) x += y;
    }
    const int b = lane + 32 * q;
    if (b < nb) {
      cum[b + 1] = base + x;
      rw[b] = r[q];
    }
    base += __shfl_sync(full, x, 31);
  }
  for (int b = lane; b <= nb; b += 32) old[b] = e[b];
  if (lane == 0) cum[0] = 0.0;
  __syncwarp();
  const double total = cum[nb];
  for (int k = 1 + lane; k < nb; k += 32) {
    const double target = total * k / nb;
    int lo = 0, hi = nb - 1;                  // cum[lo] <= target always (cum[0] = 0)
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (cum[mid] <= target) lo = mid; else hi = mid - 1;
    }
    const double frac = rw[lo] > 0.0 ? (target - cum[lo]) / rw[lo] : 0.0;
    e[k] = old[lo] + frac * (old[lo + 1] - old[lo]);
  }
  if (lane == 0) {
    e[0] = 0.0;
    e[nb] = 1.0;
  }
}

// Sum of the per-CTA partials in CTA order (deterministic for given partials).
__global__ void k_reduce(const double* __restrict__ partials, const unsigned long long* __restrict__ counters,
                         int nblocks, int nacc, double* __restrict__ totals) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nacc + 2; j += gridDim.x * blockDim.x) {
    if (j < nacc) {
      double s = 0.0;
      for (int b = 0; b < nblocks; ++b) s += partials[int64_t(b) * nacc + j];
      totals[j] = s;
    } else {
      unsigned long long c = 0;
      for (int b = 0; b < nblocks; ++b) c += counters[2 * b + (j - nacc)];
      totals[j] = double(c);
    }
  }
}

cudaError_t launch_reduce(const double* partials, const unsigned long long* counters, int nblocks, int ndim, int nbins,
                          double* totals, cudaStream_t s) {
  const int nacc = 2 + ndim * nbins;
  const int blocks = (nacc + 2 + 127) / 128;
  k_reduce<<<blocks, 128, 0, s>>>(partials, counters, nblocks, nacc, totals);
  return cudaGetLastError();
}

// Estimate of one iteration from the (possibly all-reduced) totals, and the
// refinement: warp j refines dimension j.
__global__ void k_finish(const double* __restrict__ totals, int ndim, int nbins, int64_t n, int refine,
                         double* __restrict__ edges, double* __restrict__ result) {
  __shared__ double cum[kMaxDim][65], old[kMaxDim][65], rw[kMaxDim][64];
  const int nacc = 2 + ndim * nbins;
  if (threadIdx.x == 0) {
    const double dn = double(n);
    const double I = totals[0] / dn;
    result[0] = totals[0];
    result[1] = totals[1];
    result[2] = I;
    result[3] = (totals[1] / dn - I * I) / (dn - 1.0);
    result[4] = totals[nacc];
    result[5] = totals[nacc + 1];
  }
  const int j = threadIdx.x >> 5;
  if (refine && j < ndim)
    refine_dim_warp(edges + j * (nbins + 1), totals + 2 + j * nbins, nbins, 1.5, cum[j], old[j], rw[j]);
}

cudaError_t launch_finish(const double* totals, int ndim, int nbins, int64_t n_total, int refine, double* edges,
                          double* result, cudaStream_t s) {
  if (ndim < 1 || ndim > kMaxDim || nbins < 2 || nbins > 64) return cudaErrorInvalidValue;
  k_finish<<<1, 32 * ndim, 0, s>>>(totals, ndim, nbins, n_total, refine, edges, result);
  return cudaGetLastError();
}

// FMA-pipe throughput probe: every thread runs 8 independent FMA chains, so
// the pipe, not latency, bounds it.  The result is stored only if it is
// impossible (never), which keeps the chains alive.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, float* sink) {
  T a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  const T b = T(0.999999), c = T(1e-7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == T(-1.2345)) sink[blockIdx.x] = float(s);
}

cudaError_t launch_fma_peak(int precision, int blocks, int iters, float* sink, cudaStream_t s) {
  if (precision == 0) k_fma_peak<double><<<blocks, 256, 0, s>>>(iters, sink);
  else k_fma_peak<float><<<blocks, 256, 0, s>>>(iters, sink);
  return cudaGetLastError();
}

}  // namespace mf
