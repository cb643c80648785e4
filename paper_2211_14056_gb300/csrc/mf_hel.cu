// Helicity-sampled kernels (mf_hel.cuh) for 2, 3 and 4 gluons in FP64 and
// FP32: occupancy queries and launches.
#include <cmath>

#include "mf_hel.cuh"

namespace mf {
namespace {

template <int NG, typename T> cudaError_t me_cfg(size_t* smem, int* ctas) {
  *smem = HelMem<NG, T>::warp_bytes * kWarps;
  cudaError_t e = cudaFuncSetAttribute(k_matrix_element_hel<NG, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(*smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_matrix_element_hel<NG, T>, kThreads, *smem);
}

template <int NG, typename T> cudaError_t acc_cfg(int ndim, int nbins, size_t* smem, int* ctas) {
  *smem = HelAccLayout<NG, T>::total(2 + ndim * nbins);
  cudaError_t e = cudaFuncSetAttribute(k_me_acc_hel<NG, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_me_acc_hel<NG, T>, kThreads, *smem);
}

template <int NG, typename T>
cudaError_t me_launch(const MeParams& mp, int64_t n, const double* mom, const int* hel, double* out, int grid,
                      cudaStream_t s) {
  k_matrix_element_hel<NG, T><<<grid, kThreads, HelMem<NG, T>::warp_bytes * kWarps, s>>>(mp, n, mom, hel, out);
  return cudaGetLastError();
}

template <int NG, typename T>
cudaError_t chunk_launch(const SampleParams& sp, const MeParams& mp, const double* edges, int64_t first_event,
                         int64_t n, int64_t C, void* rec_base, uint64_t seed, int iter, int accumulate,
                         double* partials, unsigned long long* counters, double* w_out, int grid, cudaStream_t s,
                         cudaEvent_t* ev, const unsigned long long* hel_T, double* hel_sq) {
  const int nacc = 2 + sp.ndim * sp.nbins;
  const size_t esm = sizeof(double) * sp.ndim * (sp.nbins + 1);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t need = (n + kThreads - 1) / kThreads;
  const int sgrid = int(need < int64_t(sms) * 16 ? need : int64_t(sms) * 16);
  RecordView<T> rec = RecordView<T>::carve(rec_base, sp.n_final, sp.ndim, C);
  e = cudaMemsetAsync(rec.count, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[0], s);
  k_sample_rec<T><<<sgrid, kThreads, esm, s>>>(sp, edges, first_event, n, seed, iter, rec, w_out);
  if (ev) cudaEventRecord(ev[1], s);
  k_me_acc_hel<NG, T><<<grid, kThreads, HelAccLayout<NG, T>::total(nacc), s>>>(
      mp, sp.ndim, sp.nbins, rec, accumulate, partials, counters, w_out, seed, iter, first_event, hel_T, hel_sq);
  if (ev) cudaEventRecord(ev[2], s);
  return cudaGetLastError();
}

// Per configuration h (lane h): the sum of the CTAs' sums in CTA order.
__global__ void k_hel_reduce(const double* __restrict__ hel_sq, int nblocks, int H, double* __restrict__ S) {
  const int h = threadIdx.x;
  if (h >= H) return;
  double acc = 0.0;
  for (int c = 0; c < nblocks; ++c) acc += hel_sq[int64_t(c) * kHelMaxConfigs + h];
  S[h] = acc;
}

// Refined thresholds (one thread, every step in configuration order and
// rounded separately, as the oracle's refinement): q_h = sqrt(p_h S_h),
// p'_h = (1 - a) q_h / sum(q) + a / H, T'_h = floor(2^32 (p'_0 + ... + p'_{h-1})).
// Unchanged when every S_h is zero.
__global__ void k_hel_refine(const double* __restrict__ S, int H, unsigned long long* __restrict__ T) {
  if (threadIdx.x != 0) return;
  double q[kHelMaxConfigs];
  double tot = 0.0;
  for (int h = 0; h < H; ++h) {
    const double ph = __dmul_rn(double(T[h + 1] - T[h]), 2.3283064365386963e-10);   // 2^-32
    q[h] = __dsqrt_rn(__dmul_rn(ph, S[h]));
    tot = __dadd_rn(tot, q[h]);
  }
  if (!(tot > 0.0)) return;
  const double om = 1.0 - kHelRefineFloor, fl = __ddiv_rn(kHelRefineFloor, double(H));
  double c = 0.0;
  unsigned long long prev = 0;
  T[0] = 0;
  for (int h = 0; h < H; ++h) {
    c = __dadd_rn(c, __dadd_rn(__dmul_rn(om, __ddiv_rn(q[h], tot)), fl));
    if (h + 1 < H) {
      unsigned long long th = (unsigned long long)floor(__dmul_rn(c, 4294967296.0));
      th = th < prev ? prev : th;
      th = th > 4294967296ull ? 4294967296ull : th;
      T[h + 1] = th;
      prev = th;
    }
  }
  T[H] = 4294967296ull;
}

}  // namespace

void hel_thresholds(const double* p, int H, unsigned long long* T) {
  double c = 0.0;
  unsigned long long prev = 0;
  T[0] = 0;
  for (int h = 0; h + 1 < H; ++h) {
    c = c + p[h];
    unsigned long long th = (unsigned long long)std::floor(c * 4294967296.0);
    th = th < prev ? prev : th;
    th = th > 4294967296ull ? 4294967296ull : th;
    T[h + 1] = th;
    prev = th;
  }
  T[H] = 4294967296ull;
}

cudaError_t launch_hel_reduce(const double* hel_sq, int nblocks, int H, double* S, cudaStream_t s) {
  k_hel_reduce<<<1, 32, 0, s>>>(hel_sq, nblocks, H, S);
  return cudaGetLastError();
}

cudaError_t launch_hel_refine(const double* S, int H, unsigned long long* T, cudaStream_t s) {
  k_hel_refine<<<1, 32, 0, s>>>(S, H, T);
  return cudaGetLastError();
}

cudaError_t hel_me_config(int ng, int precision, size_t* smem, int* ctas) {
  switch (ng) {
    case 2: return precision == 0 ? me_cfg<2, double>(smem, ctas) : me_cfg<2, float>(smem, ctas);
    case 3: return precision == 0 ? me_cfg<3, double>(smem, ctas) : me_cfg<3, float>(smem, ctas);
    case 4: return precision == 0 ? me_cfg<4, double>(smem, ctas) : me_cfg<4, float>(smem, ctas);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t hel_acc_config(int ng, int precision, int ndim, int nbins, size_t* smem, int* ctas) {
  switch (ng) {
    case 2: return precision == 0 ? acc_cfg<2, double>(ndim, nbins, smem, ctas) : acc_cfg<2, float>(ndim, nbins, smem, ctas);
    case 3: return precision == 0 ? acc_cfg<3, double>(ndim, nbins, smem, ctas) : acc_cfg<3, float>(ndim, nbins, smem, ctas);
    case 4: return precision == 0 ? acc_cfg<4, double>(ndim, nbins, smem, ctas) : acc_cfg<4, float>(ndim, nbins, smem, ctas);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_matrix_element_hel(int ng, int precision, const MeParams& mp, int64_t n, const double* mom,
                                      const int* hel, double* out, int grid, cudaStream_t s) {
  switch (ng) {
    case 2: return precision == 0 ? me_launch<2, double>(mp, n, mom, hel, out, grid, s) : me_launch<2, float>(mp, n, mom, hel, out, grid, s);
    case 3: return precision == 0 ? me_launch<3, double>(mp, n, mom, hel, out, grid, s) : me_launch<3, float>(mp, n, mom, hel, out, grid, s);
    case 4: return precision == 0 ? me_launch<4, double>(mp, n, mom, hel, out, grid, s) : me_launch<4, float>(mp, n, mom, hel, out, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_chunk_hel(int ng, int precision, const SampleParams& sp, const MeParams& mp, const double* edges,
                             int64_t first_event, int64_t n, int64_t C, void* rec_base, uint64_t seed, int iter,
                             int accumulate, double* partials, unsigned long long* counters, double* w_out, int grid,
                             cudaStream_t s, cudaEvent_t* ev, const unsigned long long* hel_T, double* hel_sq) {
#define MF_HEL_CHUNK(NG, T)                                                                                        \
  chunk_launch<NG, T>(sp, mp, edges, first_event, n, C, rec_base, seed, iter, accumulate, partials, counters, w_out, \
                      grid, s, ev, hel_T, hel_sq)
  switch (ng) {
    case 2: return precision == 0 ? MF_HEL_CHUNK(2, double) : MF_HEL_CHUNK(2, float);
    case 3: return precision == 0 ? MF_HEL_CHUNK(3, double) : MF_HEL_CHUNK(3, float);
    case 4: return precision == 0 ? MF_HEL_CHUNK(4, double) : MF_HEL_CHUNK(4, float);
    default: return cudaErrorInvalidValue;
  }
#undef MF_HEL_CHUNK
}

}  // namespace mf
