// Library-private declarations shared by the host translation units
// (mf_abi.cu, mf_mixed.cu): handle layouts and error/launch bookkeeping.
#pragma once
#include <atomic>
#include <string>
#include <vector>

#include "madflow_gb300.h"
#include "mf_kernels.cuh"

namespace mf {
namespace detail {

mf_status fail(mf_status st, const std::string& msg);
mf_status cuda_fail(cudaError_t e, const char* where);
void count_launches(int k);

#define MF_CUDA(call, where)                                 \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return mf::detail::cuda_fail(e_, where); \
  } while (0)

}  // namespace detail
}  // namespace mf

struct mf_process {
  int ng = 0, ndim = 0, precision = 0, device = 0, sms = 0;
  mf::SampleParams sp{};
  mf::MeParams mp{};
  int me_ctas = 1;
  size_t me_smem = 0;
  int ctas_override = 0;
  double g_s = 0.0, width = 0.0;   // strong coupling and top width of the descriptor
};

struct mf_grid {
  const mf_process* proc = nullptr;
  int ndim = 0, nbins = 0;
  int max_blocks = 0;
  int fused_ctas = 1;
  size_t fused_smem = 0;
  int acc_ctas = 1;            // CTAs per SM of the |M|^2-and-accumulate kernel
  size_t acc_smem = 0;
  int64_t chunk = 0;           // events per record chunk
  void* d_records = nullptr;   // per-event records of one chunk
  bool profile = false;        // record CUDA events around the kernels of each chunk
  std::vector<cudaEvent_t> ev; // 3 per chunk: before sampler, before |M|^2, after |M|^2
  int ev_used = 0;
  double* d_edges = nullptr;
  double* d_partials = nullptr;
  unsigned long long* d_counters = nullptr;
  double* d_totals = nullptr;   // [2 + ndim*nbins + 2]: sums, histogram, passing events, Newton misses
  double* d_result = nullptr;
  double* h_result = nullptr;
  std::vector<double> Ik, vark;
};

namespace mf {
namespace detail {
// Record one iteration's device result (sum w, sum w^2, I_k, sigma_k^2, passing
// events, Newton misses) on the grid and fill *out with it and the running
// inverse-variance combination.
mf_status record_iteration(mf_grid* g, const double* r, int64_t n_total, mf_result* out);
// Grow the grid's per-event record buffer to hold `events` (a configuration call).
mf_status grid_reserve(mf_grid* g, int64_t events);
int effective_ctas(const mf_process* p, int occupancy);
cudaError_t dispatch_acc_config(int ng, int prec, int ndim, int nbins, size_t* smem, int* ctas);
}  // namespace detail
}  // namespace mf
