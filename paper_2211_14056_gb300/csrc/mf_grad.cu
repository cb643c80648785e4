// Derivatives of the event weight and of the cross-section estimate with
// respect to g_s, m_t, Gamma_t and the Vegas uniforms (arXiv:2211.14056,
// Sec. 2: the custom operator lacks a derivative, "trivial to extend").
//
// mf_grad (reverse mode): per chunk, the sampling code runs with dual numbers
// Dual<B, 2> (m_t and y_0 as tangents) and writes per-event records; the
// adjoint kernel recomputes every wavefunction, current and amplitude of
// |M|^2 and sweeps back once (mf_adjoint.cuh) to d|M|^2/dp, d|M|^2/dm_t and
// d|M|^2/dGamma_t, contracts them with the record's tangents and keeps them
// per event; further sampling passes carry two more uniforms each and reuse
// the stored adjoint (the sampler is the only code they rerun).  g_s enters
// as |M|^2 ~ g_s^(2 n_gluons), so its derivative is exact.
//
// mf_grad_forward (forward mode, the cross-check): the amplitude code too
// runs with Dual<B, 2>, one pass per pair of tangents.
//
// Bins and cut decisions are piecewise constant and contribute no derivative:
// d sigma/d theta is the derivative of the estimator at fixed uniforms.
#include <cstring>

#include "mf_grad.h"

using namespace mf;
using namespace mf::detail;

static mf_status grad_entry(bool reverse, mf_process* p, const mf_grid* g, uint64_t seed, int iter, int64_t n,
                            double* sigma, double* dsigma, double* dw_dtheta, double* dw_dy, void* stream) {
  if (p == nullptr || g == nullptr || dsigma == nullptr || sigma == nullptr)
    return fail(MF_ERR_ARG, "mf_grad: null argument");
  if (g->proc != p) return fail(MF_ERR_ARG, "mf_grad: grid belongs to another process");
  if (p->kind != 0) return fail(MF_ERR_UNSUPPORTED, "mf_grad: covers the gluon-initiated processes");
  if (p->hel) return fail(MF_ERR_UNSUPPORTED, "mf_grad: differentiates the helicity sum (helicity sampling is on)");
  if (p->sp.lumi == 2) return fail(MF_ERR_UNSUPPORTED, "mf_grad: tabulated parton densities are not differentiated");
  if (n < 1) return fail(MF_ERR_ARG, "mf_grad: n must be >= 1");
  if (n > (int64_t(1) << 40)) return fail(MF_ERR_ARG, "mf_grad: n too large");
  if (iter < 0) return fail(MF_ERR_ARG, "mf_grad: iter must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  GradArgs a;
  std::memset(&a, 0, sizeof(a));
  a.sp = p->sp;
  a.sp.nbins = g->nbins;
  a.mp = p->mp;
  a.width = p->width;
  a.edges = g->d_edges;
  a.seed = seed;
  a.iter = iter;
  a.partials = g->d_partials;
  const int power = 2 * p->ng;   // |M|^2 is proportional to g_s^(2 n_gluons)
  double sums[1 + kGradTangents] = {0.0, 0.0, 0.0};
  const bool fp64 = p->precision == MF_FP64;
  mf_status st;
  switch (p->ng) {
    case 2: st = reverse ? grad_run<2, true>(fp64, p, g, a, n, dw_dtheta, dw_dy, power, sums, s)
                         : grad_run<2, false>(fp64, p, g, a, n, dw_dtheta, dw_dy, power, sums, s); break;
    case 3: st = reverse ? grad_run<3, true>(fp64, p, g, a, n, dw_dtheta, dw_dy, power, sums, s)
                         : grad_run<3, false>(fp64, p, g, a, n, dw_dtheta, dw_dy, power, sums, s); break;
    default: st = reverse ? grad_run<4, true>(fp64, p, g, a, n, dw_dtheta, dw_dy, power, sums, s)
                          : grad_run<4, false>(fp64, p, g, a, n, dw_dtheta, dw_dy, power, sums, s); break;
  }
  if (st != MF_OK) return st;
  MF_CUDA(cudaStreamSynchronize(s), "mf_grad (sync)");
  const double dn = double(n);
  *sigma = sums[0] / dn;
  dsigma[0] = power * (*sigma) / p->g_s;
  dsigma[1] = sums[1] / dn;
  dsigma[2] = sums[2] / dn;
  return MF_OK;
}

extern "C" mf_status mf_grad(mf_process* p, const mf_grid* g, uint64_t seed, int iter, int64_t n, double* sigma,
                             double* dsigma, double* dw_dtheta, double* dw_dy, void* stream) {
  return grad_entry(true, p, g, seed, iter, n, sigma, dsigma, dw_dtheta, dw_dy, stream);
}

extern "C" mf_status mf_grad_forward(mf_process* p, const mf_grid* g, uint64_t seed, int iter, int64_t n, double* sigma,
                                     double* dsigma, double* dw_dtheta, double* dw_dy, void* stream) {
  return grad_entry(false, p, g, seed, iter, n, sigma, dsigma, dw_dtheta, dw_dy, stream);
}
