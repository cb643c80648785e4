// Derivative pass, 2 gluons, reverse mode (a compile-time split of mf_grad.cu).
#include "mf_grad_impl.cuh"

namespace mf {
template <>
mf_status grad_run<2, true>(bool fp64, mf_process* p, const mf_grid* g, GradArgs& a, int64_t n,
                                   double* dw_dtheta, double* dw_dy, int power, double* sums, cudaStream_t s) {
  return fp64 ? gradimpl::grad_adjoint<2, double>(p, g, a, n, dw_dtheta, dw_dy, power, sums, s)
              : gradimpl::grad_adjoint<2, float>(p, g, a, n, dw_dtheta, dw_dy, power, sums, s);
}
}  // namespace mf
