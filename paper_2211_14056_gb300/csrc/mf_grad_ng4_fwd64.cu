// Derivative pass, 4 gluons, forward mode in FP64 (see mf_grad_ng4_fwd.cu).
#include "mf_grad_impl.cuh"

namespace mf {
mf_status grad_forward4_fp64(mf_process* p, const mf_grid* g, GradArgs& a, int64_t n, double* dw_dtheta,
                             double* dw_dy, int power, double* sums, cudaStream_t s) {
  return gradimpl::grad_forward<4, double>(p, g, a, n, dw_dtheta, dw_dy, power, sums, s);
}
}  // namespace mf
