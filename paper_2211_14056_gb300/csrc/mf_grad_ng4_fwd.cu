// Derivative pass, 4 gluons, forward mode (a compile-time split of mf_grad.cu;
// the FP64 instantiation sits in mf_grad_ng4_fwd64.cu, the largest of these
// units compiled in parallel).
#include "mf_grad_impl.cuh"

namespace mf {
mf_status grad_forward4_fp64(mf_process* p, const mf_grid* g, GradArgs& a, int64_t n, double* dw_dtheta,
                             double* dw_dy, int power, double* sums, cudaStream_t s);

template <>
mf_status grad_run<4, false>(bool fp64, mf_process* p, const mf_grid* g, GradArgs& a, int64_t n,
                                   double* dw_dtheta, double* dw_dy, int power, double* sums, cudaStream_t s) {
  return fp64 ? grad_forward4_fp64(p, g, a, n, dw_dtheta, dw_dy, power, sums, s)
              : gradimpl::grad_forward<4, float>(p, g, a, n, dw_dtheta, dw_dy, power, sums, s);
}
}  // namespace mf
