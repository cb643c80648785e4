// Declarations shared by the translation units of the derivative pass
// (mf_grad.cu and mf_grad_ng*.cu; see mf_grad.cu).
#pragma once
#include "mf_internal.h"

namespace mf {

constexpr int kGradTangents = 2;

struct GradArgs {
  SampleParams sp;
  MeParams mp;
  double width;               // Gamma_t
  const double* edges;
  int64_t first, n;           // events first .. first + n - 1 of this chunk
  uint64_t seed;
  int iter;
  TangentSeeds ts;
  int mt_slot, wt_slot;       // tangent slots of m_t and Gamma_t in the amplitude (-1: none)
  int accumulate;             // add to the partial sums (later chunks)
  double* partials;           // [gridDim.x][1 + N]: sum w, sum dw/d(slot)
  double* w_out;              // [n_total] or null: w * w_scale (indexed by global event - first of call)
  double w_scale;
  double* dw_out[kGradTangents];   // [n_total] each, or null
  // reverse mode
  int mt_tan;                 // sampler tangent slot carrying m_t (-1: none)
  double* dw_mt;              // [n_total] or null: dw/dm_t
  double* dw_wt;              // [n_total] or null: dw/dGamma_t
  double* adj;                // [C][kAdjStride]: |M|^2, d|M|^2/dp of the final particles, d|M|^2/d sqrt(s_hat)
};

// One derivative request of a gluon-initiated process with NG gluons, reverse
// (REV) or forward mode, in FP64 or FP32 (one translation unit each).
template <int NG, bool REV>
mf_status grad_run(bool fp64, mf_process* p, const mf_grid* g, GradArgs& a, int64_t n, double* dw_dtheta,
                   double* dw_dy, int power, double* sums, cudaStream_t s);

}  // namespace mf
