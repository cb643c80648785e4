// Library-private declarations shared by the host translation units
// (mf_abi.cu, mf_mixed.cu): handle layouts and error/launch bookkeeping.
#pragma once
#include <atomic>
#include <string>
#include <vector>

#include "madflow_gb300.h"
#include "mf_hel.cuh"
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
  int me_warps = 0;                // warps per CTA of the |M|^2 kernel (0: the default 4; mf_set_launch_shape)
  int hel = 0;                     // helicity sampling (mf_set_helicity_sampling): 0 sum, 1 draw from the
                                   // grid's table, 2 also accumulate the table's refinement input
  int hel_me_ctas = 0;             // CTAs per SM of k_matrix_element_hel (0: not queried yet)
  double g_s = 0.0, width = 0.0;   // strong coupling and top width of the descriptor
  int kind = 0;                    // 0: g g -> t t~ + gluons (ng = n_final), 1: u u~ -> t t~ g g,
                                   // 2: e+ e- -> mu+ mu- (ng = n_final = 2)
};

struct mf_grid {
  const mf_process* proc = nullptr;
  int ndim = 0, nbins = 0;
  int max_blocks = 0;
  int fused_ctas = 1;
  size_t fused_smem = 0;
  int acc_ctas = 1;            // CTAs per SM of the |M|^2-and-accumulate kernel
  int shape_warps = 0;         // launch shape whose occupancy shape_ctas holds (0: none yet)
  int shape_ctas = 0;
  int hel_ctas = 0;            // CTAs per SM of the helicity-sampled |M|^2 kernel (0: not queried yet)
  int hel_n = 0;               // helicity configurations drawn from (2^(NG+1); 0: no helicity table)
  unsigned long long* d_hel_T = nullptr;   // [hel_n + 1] the draw's thresholds (uniform at creation)
  double* d_hel_part = nullptr;            // [max_blocks][32] per-CTA sums of squared weights by configuration
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
  double* d_wchunk = nullptr;               // [chunk] weights of one record chunk (unweighting)
  unsigned long long* d_ucount = nullptr;   // [2] kept and overweight events (unweighting)
  std::vector<double> Ik, vark;
};

namespace mf {
// u u~ -> t t~ g g (mf_kernels_uux.cu)
cudaError_t uux_me_config(int precision, size_t* smem, int* ctas);
cudaError_t uux_acc_config(int precision, int ndim, int nbins, size_t* smem, int* ctas);
cudaError_t launch_matrix_element_uux(int precision, const MeParams& mp, int64_t n, const double* mom, double* out,
                                      int grid, cudaStream_t s);
cudaError_t launch_me_acc_uux(int precision, const MeParams& mp, int n_final, int ndim, int nbins, void* rec_base,
                              int64_t C, int accumulate, double* partials, unsigned long long* counters,
                              double* w_out, int grid, cudaStream_t s);
cudaError_t launch_chunk_uux(int precision, const SampleParams& sp, const MeParams& mp, const double* edges,
                             int64_t first_event, int64_t n, int64_t C, void* rec_base, uint64_t seed, int iter,
                             int accumulate, double* partials, unsigned long long* counters, double* w_out, int grid,
                             cudaStream_t s, cudaEvent_t* ev);
// helicity sampling for the two-quark-line channels (mf_kernels_uux.cu)
cudaError_t uux_hel_me_config(int precision, int* ctas);
cudaError_t uux_hel_acc_config(int precision, int ndim, int nbins, int* ctas);
cudaError_t launch_matrix_element_uux_hel(int precision, const MeParams& mp, int64_t n, const double* mom,
                                          const int* hel, double* out, int grid, cudaStream_t s);
cudaError_t launch_chunk_uux_hel(int precision, const SampleParams& sp, const MeParams& mp, const double* edges,
                                 int64_t first_event, int64_t n, int64_t C, void* rec_base, uint64_t seed, int iter,
                                 int accumulate, double* partials, unsigned long long* counters, double* w_out,
                                 int grid, cudaStream_t s, cudaEvent_t* ev, const unsigned long long* hel_T,
                                 double* hel_sq);
// e+ e- -> mu+ mu- (mf_kernels_ee.cu)
cudaError_t ee_me_config(int precision, size_t* smem, int* ctas);
cudaError_t ee_acc_config(int precision, int ndim, int nbins, size_t* smem, int* ctas);
cudaError_t launch_matrix_element_ee(int precision, const MeParams& mp, int64_t n, const double* mom, double* out,
                                     int grid, cudaStream_t s);
cudaError_t launch_me_acc_ee(int precision, const MeParams& mp, int n_final, int ndim, int nbins, void* rec_base,
                             int64_t C, int accumulate, double* partials, unsigned long long* counters, double* w_out,
                             int grid, cudaStream_t s);
cudaError_t launch_chunk_ee(int precision, const SampleParams& sp, const MeParams& mp, const double* edges,
                            int64_t first_event, int64_t n, int64_t C, void* rec_base, uint64_t seed, int iter,
                            int accumulate, double* partials, unsigned long long* counters, double* w_out, int grid,
                            cudaStream_t s, cudaEvent_t* ev);
namespace detail {
// Kernel-selection key of a process: the gluon count of the gluon-initiated
// processes, kUuxKey for u u~ -> t t~ g g, kEeKey for e+ e- -> mu+ mu-.
constexpr int kUuxKey = 100;
constexpr int kEeKey = 200;
inline int proc_key(const mf_process* p) { return p->kind == 1 ? kUuxKey : p->kind == 2 ? kEeKey : p->ng; }
// Record one iteration's device result (sum w, sum w^2, I_k, sigma_k^2, passing
// events, Newton misses) on the grid and fill *out with it and the running
// inverse-variance combination.
mf_status record_iteration(mf_grid* g, const double* r, int64_t n_total, mf_result* out);
// Grow the grid's per-event record buffer to hold `events` (a configuration call).
mf_status grid_reserve(mf_grid* g, int64_t events);
int effective_ctas(const mf_process* p, int occupancy);
// the device view and device of a loaded parton-density set (mf_pdf.cu)
PdfView pdf_view(const mf_pdf* p);
int pdf_device(const mf_pdf* p);
cudaError_t dispatch_acc_config(int ng, int prec, int ndim, int nbins, size_t* smem, int* ctas);
}  // namespace detail
}  // namespace mf
