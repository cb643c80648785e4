// Helicity-sampled kernels (mf_hel.cuh) for 2, 3 and 4 gluons in FP64 and
// FP32: occupancy queries and launches.
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
                         cudaEvent_t* ev) {
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
      mp, sp.ndim, sp.nbins, rec, accumulate, partials, counters, w_out, seed, iter, first_event);
  if (ev) cudaEventRecord(ev[2], s);
  return cudaGetLastError();
}

}  // namespace

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
                             cudaStream_t s, cudaEvent_t* ev) {
#define MF_HEL_CHUNK(NG, T)                                                                                        \
  chunk_launch<NG, T>(sp, mp, edges, first_event, n, C, rec_base, seed, iter, accumulate, partials, counters, w_out, \
                      grid, s, ev)
  switch (ng) {
    case 2: return precision == 0 ? MF_HEL_CHUNK(2, double) : MF_HEL_CHUNK(2, float);
    case 3: return precision == 0 ? MF_HEL_CHUNK(3, double) : MF_HEL_CHUNK(3, float);
    case 4: return precision == 0 ? MF_HEL_CHUNK(4, double) : MF_HEL_CHUNK(4, float);
    default: return cudaErrorInvalidValue;
  }
#undef MF_HEL_CHUNK
}

}  // namespace mf
