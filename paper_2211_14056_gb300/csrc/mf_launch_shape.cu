// The FP32 g g -> t t~ g g |M|^2-and-accumulate kernel at other launch shapes
// (warps per CTA), for the launch-shape study of arXiv:2211.14056 Sec. 3,
// Fig. 3 (run time of 10^6 g g -> t t~ g g events against threads per block).
// Every shape runs the same per-warp code (one lane group per event); only
// the CTA size, and with it how many CTAs share an SM's shared memory, differ.
#include "mf_internal.h"

namespace mf {

namespace {

template <int W>
cudaError_t shape_config(int ndim, int nbins, size_t* smem, int* ctas) {
  const int nacc = 2 + ndim * nbins;
  *smem = MeAccLayout<4, float, W>::total(nacc);
  cudaError_t e = cudaFuncSetAttribute(k_me_acc<4, float, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_me_acc<4, float, W>, 32 * W, *smem);
}

template <int W>
cudaError_t shape_launch(const MeParams& mp, int n_final, int ndim, int nbins, void* rec_base, int64_t C,
                         int accumulate, double* partials, unsigned long long* counters, double* w_out, int grid,
                         cudaStream_t s) {
  const int nacc = 2 + ndim * nbins;
  RecordView<float> rec = RecordView<float>::carve(rec_base, n_final, ndim, C);
  k_me_acc<4, float, W><<<grid, 32 * W, MeAccLayout<4, float, W>::total(nacc), s>>>(mp, ndim, nbins, rec, accumulate,
                                                                                      partials, counters, w_out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t me_acc_shape_config(int warps, int ndim, int nbins, size_t* smem, int* ctas) {
  switch (warps) {
    case 1: return shape_config<1>(ndim, nbins, smem, ctas);
    case 2: return shape_config<2>(ndim, nbins, smem, ctas);
    case 3: return shape_config<3>(ndim, nbins, smem, ctas);
    case 4: return shape_config<4>(ndim, nbins, smem, ctas);
    case 5: return shape_config<5>(ndim, nbins, smem, ctas);
    case 6: return shape_config<6>(ndim, nbins, smem, ctas);
    case 7: return shape_config<7>(ndim, nbins, smem, ctas);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_me_acc_shape(int warps, const MeParams& mp, int n_final, int ndim, int nbins, void* rec_base,
                                int64_t C, int accumulate, double* partials, unsigned long long* counters,
                                double* w_out, int grid, cudaStream_t s) {
  switch (warps) {
#define MF_SHAPE(W) \
    case W: return shape_launch<W>(mp, n_final, ndim, nbins, rec_base, C, accumulate, partials, counters, w_out, grid, s);
    MF_SHAPE(1) MF_SHAPE(2) MF_SHAPE(3) MF_SHAPE(4) MF_SHAPE(5) MF_SHAPE(6) MF_SHAPE(7)
#undef MF_SHAPE
  }
  return cudaErrorInvalidValue;
}

}  // namespace mf
