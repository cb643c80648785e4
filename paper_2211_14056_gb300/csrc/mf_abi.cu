// C ABI of the library (declarations and their documentation: include/madflow_gb300.h).
// Host side only: argument checks, handle lifetime, launch sizing, the Vegas
// iteration record and its combination (Lepage's inverse-variance mean).
#include <algorithm>
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mf_internal.h"
#include "mf_gen_uux.cuh"

using namespace mf;

namespace mf {
namespace detail {

thread_local std::string g_err;
std::atomic<int64_t> g_launches{0};

mf_status fail(mf_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

mf_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return MF_ERR_CUDA;
}

void count_launches(int k) { g_launches.fetch_add(k); }

}  // namespace detail
}  // namespace mf

using namespace mf::detail;

namespace {

int factorial(int n) { return n <= 1 ? 1 : n * factorial(n - 1); }

// events per record chunk of the two-kernel iteration (records: ~90 B/event
// in FP32, ~160 B/event in FP64)
constexpr int64_t kRecordChunk = int64_t(1) << 20;

// colourless process: the 1 x 1 matrix 1
const int kNoColour[1] = {1};

const int* lib_colour(int key, int* den) {
  switch (key) {
    case 2: *den = kColourDen2; return kColourNum2;
    case 3: *den = kColourDen3; return kColourNum3;
    case 4: *den = kColourDen4; return kColourNum4;
    case mf::detail::kUuxKey: *den = kUuxColourDen; return kUuxColourNum;
    case mf::detail::kEeKey: *den = 1; return kNoColour;
  }
  return nullptr;
}

}  // namespace

namespace mf {
namespace detail {
cudaError_t dispatch_acc_config(int ng, int prec, int ndim, int nbins, size_t* smem, int* ctas) {
  const int p = prec == MF_FP64 ? 0 : 1;
  switch (ng) {
    case 2: return me_acc_config<2>(p, ndim, nbins, smem, ctas);
    case 3: return me_acc_config<3>(p, ndim, nbins, smem, ctas);
    case 4: return me_acc_config<4>(p, ndim, nbins, smem, ctas);
    case kUuxKey: return uux_acc_config(p, ndim, nbins, smem, ctas);
    case kEeKey: return ee_acc_config(p, ndim, nbins, smem, ctas);
  }
  return cudaErrorInvalidValue;
}

int effective_ctas(const mf_process* p, int occupancy) {
  if (p->ctas_override > 0 && p->ctas_override < occupancy) return p->ctas_override;
  return occupancy < 1 ? 1 : occupancy;
}
}  // namespace detail
}  // namespace mf

namespace {

cudaError_t dispatch_fused_config(int ng, int prec, int ndim, int nbins, size_t* smem, int* ctas) {
  const int p = prec == MF_FP64 ? 0 : 1;
  switch (ng) {
    case 2: return fused_config<2>(p, ndim, nbins, smem, ctas);
    case 3: return fused_config<3>(p, ndim, nbins, smem, ctas);
    case 4: return fused_config<4>(p, ndim, nbins, smem, ctas);
  }
  return cudaErrorInvalidValue;
}

cudaError_t dispatch_me_config(int ng, int prec, size_t* smem, int* ctas) {
  const int p = prec == MF_FP64 ? 0 : 1;
  switch (ng) {
    case 2: return me_config<2>(p, smem, ctas);
    case 3: return me_config<3>(p, smem, ctas);
    case 4: return me_config<4>(p, smem, ctas);
    case mf::detail::kUuxKey: return uux_me_config(p, smem, ctas);
    case mf::detail::kEeKey: return ee_me_config(p, smem, ctas);
  }
  return cudaErrorInvalidValue;
}


}  // namespace

namespace mf {
namespace detail {
mf_status record_iteration(mf_grid* g, const double* r, int64_t n_total, mf_result* out) {
  out->I_k = r[2];
  out->sigma_k = std::sqrt(r[3] > 0 ? r[3] : 0.0);
  out->n_events = n_total;
  out->n_pass = int64_t(r[4]);
  out->n_newton_fail = int64_t(r[5]);
  if (!(r[3] > 0) || !std::isfinite(r[2]) || !std::isfinite(r[3])) {
    // not recorded: the inverse-variance combination cannot weigh it, and the
    // recorded history stays one that mf_grid_set_history accepts
    out->iterations = int(g->Ik.size());
    out->I = out->sigma = out->chi2dof = NAN;
    return fail(MF_ERR_ARG, "mf_vegas_finish: the iteration has zero variance (or a non-finite estimate); "
                            "combination undefined, iteration not recorded");
  }
  g->Ik.push_back(r[2]);
  g->vark.push_back(r[3]);
  out->iterations = int(g->Ik.size());
  double sw = 0, swi = 0;
  for (size_t k = 0; k < g->Ik.size(); ++k) {
    sw += 1.0 / g->vark[k];
    swi += g->Ik[k] / g->vark[k];
  }
  out->I = swi / sw;
  out->sigma = 1.0 / std::sqrt(sw);
  double chi = 0;
  for (size_t k = 0; k < g->Ik.size(); ++k) chi += (g->Ik[k] - out->I) * (g->Ik[k] - out->I) / g->vark[k];
  out->chi2dof = g->Ik.size() > 1 ? chi / double(g->Ik.size() - 1) : 0.0;
  return out->n_newton_fail > 0 ? MF_WARN_NEWTON : MF_OK;
}
mf_status grid_reserve(mf_grid* g, int64_t events) {
  if (events <= g->chunk) return MF_OK;
  void* buf = nullptr;
  double* wbuf = nullptr;
  MF_CUDA(cudaMalloc(&buf, record_bytes(g->proc->precision == MF_FP64 ? 0 : 1, g->proc->sp.n_final, g->ndim, events)),
          "grid_reserve");
  cudaError_t e = cudaMalloc(&wbuf, sizeof(double) * events);
  if (e != cudaSuccess) {
    cudaFree(buf);
    return cuda_fail(e, "grid_reserve");
  }
  cudaFree(g->d_records);
  cudaFree(g->d_wchunk);
  g->d_records = buf;
  g->d_wchunk = wbuf;
  g->chunk = events;
  return MF_OK;
}
}  // namespace detail
}  // namespace mf

extern "C" {

const char* mf_last_error(void) { return g_err.c_str(); }

int64_t mf_kernel_launches(void) { return g_launches.load(); }

mf_status mf_init_process(const mf_process_desc* d, mf_process** out) {
  if (d == nullptr || out == nullptr) return fail(MF_ERR_ARG, "mf_init_process: null argument");
  *out = nullptr;
  int ng = 0, kind = 0, chan = 0;
  switch (d->process_id) {
    case MF_PROC_GG_TTX: ng = 2; break;
    case MF_PROC_GG_TTXG: ng = 3; break;
    case MF_PROC_GG_TTXGG: ng = 4; break;
    case MF_PROC_UUX_TTXGG: ng = 4; kind = 1; chan = kChanQQB; break;
    case MF_PROC_EE_MUMU: ng = 2; kind = 2; break;
    case MF_PROC_UXU_TTXGG: ng = 4; kind = 1; chan = kChanQBQ; break;
    case MF_PROC_UG_TTXGU: ng = 4; kind = 1; chan = kChanQG; break;
    case MF_PROC_GU_TTXGU: ng = 4; kind = 1; chan = kChanGQ; break;
    case MF_PROC_UXG_TTXGUX: ng = 4; kind = 1; chan = kChanQBG; break;
    case MF_PROC_GUX_TTXGUX: ng = 4; kind = 1; chan = kChanGQB; break;
    default: return fail(MF_ERR_UNSUPPORTED, "mf_init_process: unknown process_id");
  }
  const bool quark_gluon = kind == 1 && chan >= kChanQG;   // one final gluon and a final quark
  const bool qed = kind == 2;
  const int key = kind == 1 ? kUuxKey : qed ? kEeKey : ng;
  const int nflow = kind == 1 ? kUuxFlows : qed ? 1 : factorial(ng);
  if (d->n_ext != ng + 2) return fail(MF_ERR_ARG, "mf_init_process: n_ext does not match the process");
  if (d->masses == nullptr) return fail(MF_ERR_ARG, "mf_init_process: masses is null");
  const double mt = qed ? 0.0 : d->masses[2];
  for (int i = 0; i < d->n_ext; ++i) {
    const bool top = !qed && (i == 2 || i == 3);
    if (!std::isfinite(d->masses[i]) || (top ? !(d->masses[i] > 0) : d->masses[i] != 0.0))
      return fail(MF_ERR_ARG, qed ? "mf_init_process: the leptons of e+ e- -> mu+ mu- are massless"
                                  : "mf_init_process: masses must be (0, 0, m_t, m_t, 0, ...) with m_t > 0");
  }
  if (d->masses[3] != d->masses[2]) return fail(MF_ERR_ARG, "mf_init_process: top and antitop masses differ");
  if (!(d->top_width >= 0) || !std::isfinite(d->top_width)) return fail(MF_ERR_ARG, "mf_init_process: bad top_width");
  if (qed) {
    if (!(d->e_qed > 0) || !std::isfinite(d->e_qed)) return fail(MF_ERR_ARG, "mf_init_process: bad e_qed");
    if (d->lumi != 0) return fail(MF_ERR_ARG, "mf_init_process: e+ e- -> mu+ mu- runs at a fixed energy (lumi = 0)");
  } else if (!(d->g_s > 0) || !std::isfinite(d->g_s)) {
    return fail(MF_ERR_ARG, "mf_init_process: bad g_s");
  }
  if (d->precision != MF_FP64 && d->precision != MF_FP32 && d->precision != MF_FP32_TC)
    return fail(MF_ERR_ARG, "mf_init_process: bad precision");
  // colour matrix: must be the library's exact trace-basis matrix
  if (kind != 0 && d->precision == MF_FP32_TC)
    return fail(MF_ERR_UNSUPPORTED, "mf_init_process: the tensor-core colour sum covers the gluon-initiated processes");
  if (d->n_flow != nflow) return fail(MF_ERR_COLOUR, "mf_init_process: n_flow does not match the process's colour basis");
  if (d->colour_num == nullptr || d->colour_den <= 0) return fail(MF_ERR_COLOUR, "mf_init_process: colour matrix missing");
  int lden = 1;
  const int* lnum = lib_colour(key, &lden);
  const int nf = d->n_flow;
  for (int a = 0; a < nf; ++a)
    for (int b = 0; b < nf; ++b) {
      const int64_t x = d->colour_num[a * nf + b];
      if (x != d->colour_num[b * nf + a]) return fail(MF_ERR_COLOUR, "mf_init_process: colour matrix not symmetric");
      // x / den == lnum / lden  <=>  x * lden == lnum * den
      if (x * int64_t(lden) != int64_t(lnum[a * nf + b]) * d->colour_den)
        return fail(MF_ERR_COLOUR, "mf_init_process: colour matrix differs from the process's trace-basis matrix");
      if (std::abs(lnum[a * nf + b]) > 2048)
        return fail(MF_ERR_COLOUR, "mf_init_process: scaled colour matrix is not TF32-exact");
    }
  if (!(d->sqrt_s > 2 * mt) || !std::isfinite(d->sqrt_s))
    return fail(MF_ERR_ARG, qed ? "mf_init_process: sqrt_s must be > 0" : "mf_init_process: sqrt_s must exceed 2 m_t");
  if (d->lumi != 0 && d->lumi != 1 && d->lumi != 2) return fail(MF_ERR_ARG, "mf_init_process: lumi must be 0, 1 or 2");
  if (d->lumi == 1 && !(d->lumi_N > 0 && d->lumi_b >= 0 && std::isfinite(d->lumi_a)))
    return fail(MF_ERR_ARG, "mf_init_process: bad luminosity parameters");
  PdfView pview{};
  if (d->lumi == 2) {
    if (d->pdf == nullptr || d->pairs == nullptr || d->n_pairs < 1 || d->n_pairs > kMaxPdfPairs)
      return fail(MF_ERR_ARG, "mf_init_process: lumi = 2 needs a parton-density set and 1..8 parton pairs");
    if (!(d->mu_f > 0) || !std::isfinite(d->mu_f)) return fail(MF_ERR_ARG, "mf_init_process: mu_f must be > 0");
    pview = pdf_view(d->pdf);
    for (int k = 0; k < 2 * d->n_pairs; ++k)
      if (d->pairs[k] < 0 || d->pairs[k] >= pview.nflav)
        return fail(MF_ERR_ARG, "mf_init_process: a parton pair names a flavour outside the set");
    int dev = 0;
    cudaError_t ed = cudaGetDevice(&dev);
    if (ed != cudaSuccess) return cuda_fail(ed, "mf_init_process");
    if (dev != pdf_device(d->pdf)) return fail(MF_ERR_ARG, "mf_init_process: the set lives on another device");
  }
  if (!(d->pt_cut_g >= 0) || !(d->dr_cut_gg >= 0)) return fail(MF_ERR_ARG, "mf_init_process: cuts must be >= 0");

  mf_process* p = new mf_process();
  p->ng = ng;
  p->kind = kind;
  p->precision = d->precision;
  const int n = ng;   // final-state particles: t, tbar and ng - 2 gluons (mu-, mu+ for e+ e-)
  p->ndim = 3 * n - 4 + (d->lumi ? 2 : 0);
  SampleParams& sp = p->sp;
  sp.n_final = n;
  sp.ndim = p->ndim;
  sp.nbins = 50;
  sp.lumi = d->lumi;
  sp.sqrt_s = d->sqrt_s;
  sp.tau0 = 4.0 * mt * mt / (d->sqrt_s * d->sqrt_s);
  sp.log_tau0 = std::log(sp.tau0);
  sp.lumi_N = d->lumi_N;
  sp.lumi_a = d->lumi_a;
  sp.lumi_b = d->lumi_b;
  sp.mt = mt;
  sp.pt_cut2 = d->pt_cut_g * d->pt_cut_g;
  sp.dr_cut2 = d->dr_cut_gg * d->dr_cut_gg;
  const double pi = 3.14159265358979323846;
  sp.phi_const = std::pow(2 * pi, 4 - 3 * n) * std::pow(pi / 2, n - 1) / (factorial(n - 1) * factorial(n - 2));
  if (d->lumi == 2) {
    sp.pdf = pview;
    sp.npairs = d->n_pairs;
    for (int k = 0; k < d->n_pairs; ++k) {
      sp.pairs[k][0] = uint8_t(d->pairs[2 * k]);
      sp.pairs[k][1] = uint8_t(d->pairs[2 * k + 1]);
    }
    sp.ln_muf2_S = 2.0 * std::log(d->mu_f) + 2.0 * std::log(d->sqrt_s);
  }
  MeParams& mp = p->mp;
  mp.mt = mt;
  mp.mw = qed ? 0.0 : mt * d->top_width;
  mp.colour_tc = d->precision == MF_FP32_TC ? 1 : 0;
  mp.chan = chan;
  p->g_s = d->g_s;
  p->width = d->top_width;
  const int sid = quark_gluon ? 1 : factorial(ng - 2);   // identical final-state gluons
  // spin x colour states of the initial partons: q q~ 4*9, q g 4*24, e+ e- 4, g g 4*64
  const double average = quark_gluon ? 96.0 : kind == 1 ? 36.0 : qed ? 4.0 : 256.0;
  mp.norm = qed ? std::pow(d->e_qed, 4) / average : std::pow(d->g_s, 2 * ng) / (average * sid * lden);

  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
  if (e == cudaSuccess) e = dispatch_me_config(key, p->precision, &p->me_smem, &p->me_ctas);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "mf_init_process");
  }
  if (p->me_ctas < 1) {
    delete p;
    return fail(MF_ERR_CUDA, "mf_init_process: matrix-element kernel does not fit on an SM");
  }
  *out = p;
  g_err.clear();
  return MF_OK;
}

mf_status mf_destroy_process(mf_process* p) {
  delete p;
  return MF_OK;
}

mf_status mf_process_ndim(const mf_process* p, int* ndim) {
  if (p == nullptr || ndim == nullptr) return fail(MF_ERR_ARG, "mf_process_ndim: null argument");
  *ndim = p->ndim;
  return MF_OK;
}

mf_status mf_set_ctas_per_sm(mf_process* p, int c) {
  if (p == nullptr || c < 0) return fail(MF_ERR_ARG, "mf_set_ctas_per_sm: bad argument");
  p->ctas_override = c;
  return MF_OK;
}

mf_status mf_set_launch_shape(mf_process* p, int warps_per_cta, int* max_ctas_per_sm) {
  if (p == nullptr || warps_per_cta < 0 || warps_per_cta > 7)
    return fail(MF_ERR_ARG, "mf_set_launch_shape: warps_per_cta must be in [0, 7]");
  if (warps_per_cta > 0 && (p->kind != 0 || p->ng != 4 || p->precision == MF_FP64))
    return fail(MF_ERR_UNSUPPORTED, "mf_set_launch_shape: launch shapes exist for g g -> t t~ g g in FP32");
  if (warps_per_cta > 0) {
    size_t smem = 0;
    int ctas = 0;
    MF_CUDA(me_acc_shape_config(warps_per_cta, p->ndim, 50, &smem, &ctas), "mf_set_launch_shape");
    if (ctas < 1)
      return fail(MF_ERR_UNSUPPORTED, "mf_set_launch_shape: " + std::to_string(warps_per_cta) + " warps (" +
                                          std::to_string(smem) + " bytes of shared memory) do not fit on an SM");
    if (max_ctas_per_sm != nullptr) *max_ctas_per_sm = ctas;
  } else if (max_ctas_per_sm != nullptr) {
    size_t smem = 0;
    MF_CUDA(dispatch_acc_config(proc_key(p), p->precision, p->ndim, 50, &smem, max_ctas_per_sm), "mf_set_launch_shape");
  }
  p->me_warps = warps_per_cta;
  return MF_OK;
}

mf_status mf_set_helicity_sampling(mf_process* p, int on) {
  if (p == nullptr || on < 0 || on > 2) return fail(MF_ERR_ARG, "mf_set_helicity_sampling: need a process and on = 0, 1 or 2");
  if (on && (p->kind == 2 || p->precision == MF_FP32_TC))
    return fail(MF_ERR_UNSUPPORTED, "mf_set_helicity_sampling: covers the g g and p p -> t t~ + jets processes "
                                    "in MF_FP64 or MF_FP32");
  if (on && p->hel_me_ctas == 0) {
    size_t smem = 0;
    int ctas = 0;
    MF_CUDA(p->kind == 1 ? uux_hel_me_config(p->precision == MF_FP64 ? 0 : 1, &ctas)
                         : hel_me_config(p->ng, p->precision == MF_FP64 ? 0 : 1, &smem, &ctas),
            "mf_set_helicity_sampling");
    if (ctas < 1) return fail(MF_ERR_UNSUPPORTED, "mf_set_helicity_sampling: the kernel does not fit on an SM");
    p->hel_me_ctas = ctas;
  }
  p->hel = on;
  return MF_OK;
}

mf_status mf_grid_create(const mf_process* p, int nbins, mf_grid** out) {
  if (p == nullptr || out == nullptr) return fail(MF_ERR_ARG, "mf_grid_create: null argument");
  if (nbins < 2 || nbins > 64) return fail(MF_ERR_ARG, "mf_grid_create: nbins must be in [2, 64]");
  *out = nullptr;
  mf_grid* g = new mf_grid();
  g->proc = p;
  g->ndim = p->ndim;
  g->nbins = nbins;
  // the fused kernel (allocation-free entry point) exists for the gluon-initiated processes
  cudaError_t e = cudaSuccess;
  if (p->kind == 0) {
    e = dispatch_fused_config(p->ng, p->precision, g->ndim, nbins, &g->fused_smem, &g->fused_ctas);
    if (e == cudaSuccess && g->fused_ctas < 1) e = cudaErrorInvalidConfiguration;
  } else {
    g->fused_ctas = 0;
  }
  if (e == cudaSuccess) e = dispatch_acc_config(proc_key(p), p->precision, g->ndim, nbins, &g->acc_smem, &g->acc_ctas);
  if (e == cudaSuccess && g->acc_ctas < 1) e = cudaErrorInvalidConfiguration;
  // CTA partials: room for the largest persistent grid any launch shape uses
  // (at most 8 resident warps per SM, one warp per CTA)
  const int most = std::max(std::max(g->fused_ctas, g->acc_ctas), 8);
  g->max_blocks = p->sms * most;
  g->chunk = kRecordChunk;
  std::vector<double> edges(size_t(g->ndim) * (nbins + 1));
  for (int j = 0; j < g->ndim; ++j)
    for (int b = 0; b <= nbins; ++b) edges[size_t(j) * (nbins + 1) + b] = double(b) / nbins;
  const size_t nacc = 2 + size_t(g->ndim) * nbins;
  if (e == cudaSuccess) e = cudaMalloc(&g->d_edges, sizeof(double) * edges.size());
  if (e == cudaSuccess) e = cudaMalloc(&g->d_partials, sizeof(double) * nacc * g->max_blocks);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_counters, sizeof(unsigned long long) * 2 * g->max_blocks);
  // totals: the Vegas sums, the counters, then (adaptive helicity sampling)
  // the configurations' sums of squared weights
  if (e == cudaSuccess) e = cudaMalloc(&g->d_totals, sizeof(double) * (nacc + 2 + kHelMaxConfigs));
  if (e == cudaSuccess)
    e = cudaMalloc(&g->d_records, record_bytes(p->precision == MF_FP64 ? 0 : 1, p->sp.n_final, g->ndim, g->chunk));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_result, sizeof(double) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_wchunk, sizeof(double) * g->chunk);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_ucount, sizeof(unsigned long long) * 2);
  if (e == cudaSuccess && (p->kind == 0 || p->kind == 1)) {
    // the helicity table: uniform thresholds over the 2^(NG+1) configurations
    // of the gluon-initiated processes, the 32 of the two-quark-line ones
    g->hel_n = p->kind == 0 ? 2 << p->ng : 32;
    std::vector<unsigned long long> T(g->hel_n + 1);
    for (int h = 0; h <= g->hel_n; ++h) T[h] = (unsigned long long)h * (4294967296ull / g->hel_n);
    e = cudaMalloc(&g->d_hel_T, sizeof(unsigned long long) * (g->hel_n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_hel_part, sizeof(double) * kHelMaxConfigs * g->max_blocks);
    if (e == cudaSuccess)
      e = cudaMemcpy(g->d_hel_T, T.data(), sizeof(unsigned long long) * T.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMallocHost(&g->h_result, sizeof(double) * 8);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_edges, edges.data(), sizeof(double) * edges.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    mf_grid_destroy(g);
    return cuda_fail(e, "mf_grid_create");
  }
  *out = g;
  return MF_OK;
}

mf_status mf_grid_destroy(mf_grid* g) {
  if (g == nullptr) return MF_OK;
  cudaFree(g->d_edges);
  cudaFree(g->d_partials);
  cudaFree(g->d_records);
  for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
  cudaFree(g->d_counters);
  cudaFree(g->d_totals);
  cudaFree(g->d_result);
  cudaFree(g->d_wchunk);
  cudaFree(g->d_ucount);
  cudaFree(g->d_hel_T);
  cudaFree(g->d_hel_part);
  cudaFreeHost(g->h_result);
  delete g;
  return MF_OK;
}

mf_status mf_grid_get(const mf_grid* g, double* h) {
  if (g == nullptr || h == nullptr) return fail(MF_ERR_ARG, "mf_grid_get: null argument");
  MF_CUDA(cudaMemcpy(h, g->d_edges, sizeof(double) * g->ndim * (g->nbins + 1), cudaMemcpyDeviceToHost), "mf_grid_get");
  return MF_OK;
}

mf_status mf_grid_set(mf_grid* g, const double* h) {
  if (g == nullptr || h == nullptr) return fail(MF_ERR_ARG, "mf_grid_set: null argument");
  for (int j = 0; j < g->ndim; ++j) {
    const double* e = h + size_t(j) * (g->nbins + 1);
    if (e[0] != 0.0 || e[g->nbins] != 1.0) return fail(MF_ERR_ARG, "mf_grid_set: a row does not span [0, 1]");
    for (int b = 0; b < g->nbins; ++b)
      if (!(e[b + 1] > e[b])) return fail(MF_ERR_ARG, "mf_grid_set: edges must increase strictly");
  }
  MF_CUDA(cudaMemcpy(g->d_edges, h, sizeof(double) * g->ndim * (g->nbins + 1), cudaMemcpyHostToDevice), "mf_grid_set");
  return MF_OK;
}

mf_status mf_grid_reset(mf_grid* g) {
  if (g == nullptr) return fail(MF_ERR_ARG, "mf_grid_reset: null argument");
  g->Ik.clear();
  g->vark.clear();
  return MF_OK;
}

mf_status mf_grid_history(const mf_grid* g, int* count, double* I_k, double* var_k) {
  if (g == nullptr || count == nullptr) return fail(MF_ERR_ARG, "mf_grid_history: null argument");
  const int have = int(g->Ik.size());
  if (I_k == nullptr && var_k == nullptr) {
    *count = have;
    return MF_OK;
  }
  if (I_k == nullptr || var_k == nullptr) return fail(MF_ERR_ARG, "mf_grid_history: need both arrays or neither");
  if (*count < have) return fail(MF_ERR_ARG, "mf_grid_history: arrays shorter than the record");
  for (int k = 0; k < have; ++k) {
    I_k[k] = g->Ik[size_t(k)];
    var_k[k] = g->vark[size_t(k)];
  }
  *count = have;
  return MF_OK;
}

mf_status mf_grid_set_history(mf_grid* g, int count, const double* I_k, const double* var_k) {
  if (g == nullptr || count < 0 || (count > 0 && (I_k == nullptr || var_k == nullptr)))
    return fail(MF_ERR_ARG, "mf_grid_set_history: bad argument");
  for (int k = 0; k < count; ++k)
    if (!std::isfinite(I_k[k]) || !(var_k[k] > 0) || !std::isfinite(var_k[k]))
      return fail(MF_ERR_ARG, "mf_grid_set_history: estimates must be finite and variances > 0");
  g->Ik.assign(I_k, I_k + count);
  g->vark.assign(var_k, var_k + count);
  return MF_OK;
}

mf_status mf_sample(mf_process* p, const mf_grid* g, uint64_t seed, int iter, int64_t n, double* momenta,
                    double* weight_ps, uint8_t* bins, void* stream) {
  if (p == nullptr || g == nullptr || n < 0) return fail(MF_ERR_ARG, "mf_sample: bad argument");
  if (g->proc != p) return fail(MF_ERR_ARG, "mf_sample: grid belongs to another process");
  if (n == 0) return MF_OK;
  SampleParams sp = p->sp;
  sp.nbins = g->nbins;
  MF_CUDA(launch_sample(sp, g->d_edges, n, seed, iter, momenta, weight_ps, bins, (cudaStream_t)stream), "mf_sample");
  g_launches.fetch_add(1);
  return MF_OK;
}

mf_status mf_uniforms(uint64_t seed, int iter, int64_t first_event, int64_t n, int ndim, double* y, void* stream) {
  if (n < 0 || first_event < 0 || ndim < 1 || ndim > kMaxDim) return fail(MF_ERR_ARG, "mf_uniforms: bad argument");
  if (n == 0) return MF_OK;
  if (y == nullptr) return fail(MF_ERR_ARG, "mf_uniforms: null buffer");
  MF_CUDA(launch_uniforms(seed, iter, first_event, n, ndim, y, (cudaStream_t)stream), "mf_uniforms");
  g_launches.fetch_add(1);
  return MF_OK;
}

mf_status mf_matrix_element(mf_process* p, int64_t n, const double* momenta, double* me2, void* stream) {
  if (p == nullptr || n < 0) return fail(MF_ERR_ARG, "mf_matrix_element: bad argument");
  if (n == 0) return MF_OK;
  if (momenta == nullptr || me2 == nullptr) return fail(MF_ERR_ARG, "mf_matrix_element: null buffer");
  const int epb = p->kind == 1 ? kWarps : p->kind == 2 ? kThreads : kWarps * (32 / (2 << p->ng));   // events per CTA pass
  const int64_t need = (n + epb - 1) / epb;
  const int64_t cap = int64_t(p->sms) * effective_ctas(p, p->me_ctas);
  const int grid = int(need < cap ? need : cap);
  cudaError_t e;
  switch (proc_key(p)) {
    case kUuxKey: e = launch_matrix_element_uux(p->precision == MF_FP64 ? 0 : 1, p->mp, n, momenta, me2, grid, (cudaStream_t)stream); break;
    case kEeKey: e = launch_matrix_element_ee(p->precision == MF_FP64 ? 0 : 1, p->mp, n, momenta, me2, grid, (cudaStream_t)stream); break;
    case 2: e = launch_matrix_element<2>(p->precision == MF_FP64 ? 0 : 1, p->mp, n, momenta, me2, grid, (cudaStream_t)stream); break;
    case 3: e = launch_matrix_element<3>(p->precision == MF_FP64 ? 0 : 1, p->mp, n, momenta, me2, grid, (cudaStream_t)stream); break;
    default: e = launch_matrix_element<4>(p->precision == MF_FP64 ? 0 : 1, p->mp, n, momenta, me2, grid, (cudaStream_t)stream); break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "mf_matrix_element");
  g_launches.fetch_add(1);
  return MF_OK;
}

mf_status mf_matrix_element_hel(mf_process* p, int64_t n, const double* momenta, const int32_t* hel, double* me2,
                                void* stream) {
  if (p == nullptr || n < 0) return fail(MF_ERR_ARG, "mf_matrix_element_hel: bad argument");
  if (p->kind == 2 || p->precision == MF_FP32_TC)
    return fail(MF_ERR_UNSUPPORTED, "mf_matrix_element_hel: covers the g g and p p -> t t~ + jets processes "
                                    "in MF_FP64 or MF_FP32");
  if (n == 0) return MF_OK;
  if (momenta == nullptr || hel == nullptr || me2 == nullptr) return fail(MF_ERR_ARG, "mf_matrix_element_hel: null buffer");
  const int prec = p->precision == MF_FP64 ? 0 : 1;
  if (p->hel_me_ctas == 0) {
    size_t smem = 0;
    int ctas = 0;
    MF_CUDA(p->kind == 1 ? uux_hel_me_config(prec, &ctas) : hel_me_config(p->ng, prec, &smem, &ctas),
            "mf_matrix_element_hel");
    if (ctas < 1) return fail(MF_ERR_UNSUPPORTED, "mf_matrix_element_hel: the kernel does not fit on an SM");
    p->hel_me_ctas = ctas;
  }
  const int epb = p->kind == 1 ? kThreads : kWarps * kHelEPW;   // events per CTA pass
  const int64_t need = (n + epb - 1) / epb;
  const int64_t cap = int64_t(p->sms) * effective_ctas(p, p->hel_me_ctas);
  const int grid = int(need < cap ? need : cap);
  if (p->kind == 1)
    MF_CUDA(launch_matrix_element_uux_hel(prec, p->mp, n, momenta, hel, me2, grid, (cudaStream_t)stream),
            "mf_matrix_element_hel");
  else
    MF_CUDA(launch_matrix_element_hel(p->ng, prec, p->mp, n, momenta, hel, me2, grid, (cudaStream_t)stream),
            "mf_matrix_element_hel");
  g_launches.fetch_add(1);
  return MF_OK;
}

// CTAs per SM of the helicity-sampled |M|^2-and-accumulate kernel for a grid's
// binning, queried once per grid
static mf_status hel_grid_ctas(const mf_process* p, mf_grid* g) {
  if (g->hel_ctas > 0) return MF_OK;
  size_t smem = 0;
  int ctas = 0;
  MF_CUDA(p->kind == 1 ? uux_hel_acc_config(p->precision == MF_FP64 ? 0 : 1, g->ndim, g->nbins, &ctas)
                       : hel_acc_config(p->ng, p->precision == MF_FP64 ? 0 : 1, g->ndim, g->nbins, &smem, &ctas),
          "helicity-sampled kernel configuration");
  if (ctas < 1) return fail(MF_ERR_UNSUPPORTED, "the helicity-sampled kernel does not fit on an SM");
  g->hel_ctas = ctas;
  return MF_OK;
}

mf_status mf_vegas_accumulate(mf_process* p, mf_grid* g, uint64_t seed, int iter, int64_t first_event, int64_t n,
                              double* weights, void* stream) {
  if (p == nullptr || g == nullptr) return fail(MF_ERR_ARG, "mf_vegas_accumulate: null argument");
  if (g->proc != p) return fail(MF_ERR_ARG, "mf_vegas_accumulate: grid belongs to another process");
  if (n < 1 || first_event < 0) return fail(MF_ERR_ARG, "mf_vegas_accumulate: need n >= 1 and first_event >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  SampleParams sp = p->sp;
  sp.nbins = g->nbins;
  const int prec = p->precision == MF_FP64 ? 0 : 1;
  const int warps = p->me_warps > 0 ? p->me_warps : kWarps;
  int acc_ctas = g->acc_ctas;
  if (p->me_warps > 0) {
    if (g->shape_warps != p->me_warps) {
      size_t smem = 0;
      int ctas = 0;
      MF_CUDA(me_acc_shape_config(p->me_warps, g->ndim, g->nbins, &smem, &ctas), "mf_vegas_accumulate (launch shape)");
      if (ctas < 1) return fail(MF_ERR_UNSUPPORTED, "mf_vegas_accumulate: the launch shape does not fit on an SM");
      g->shape_warps = p->me_warps;
      g->shape_ctas = ctas;
    }
    acc_ctas = g->shape_ctas;
  }
  if (p->hel) {
    const mf_status st = hel_grid_ctas(p, g);
    if (st != MF_OK) return st;
    acc_ctas = g->hel_ctas;
  }
  const int64_t cap = std::min<int64_t>(int64_t(p->sms) * effective_ctas(p, acc_ctas), g->max_blocks);
  int grid = 0;
  if (g->profile) {
    const size_t need = size_t(3) * size_t((n + g->chunk - 1) / g->chunk);
    while (g->ev.size() < need) {
      cudaEvent_t e;
      MF_CUDA(cudaEventCreate(&e), "mf_vegas_accumulate (profiling events)");
      g->ev.push_back(e);
    }
    g->ev_used = int(need);
  }
  // chunks of the record buffer: sample the chunk, then |M|^2 + accumulate;
  // the CTA partials of every chunk add up in place
  for (int64_t done = 0, k = 0; done < n; done += g->chunk, ++k) {
    const int64_t m = std::min(g->chunk, n - done);
    const int64_t warps_needed = (m + 31) / 32;
    const int64_t ctas_needed = (warps_needed + warps - 1) / warps;
    if (k == 0) grid = int(std::min(cap, std::max<int64_t>(ctas_needed, 1)));
    double* w = weights ? weights + done : nullptr;
    cudaEvent_t* evk = g->profile ? &g->ev[size_t(3) * k] : nullptr;
    cudaError_t e;
    if (p->hel) {
      double* hsq = p->hel == 2 ? g->d_hel_part : nullptr;
      e = p->kind == 1
              ? launch_chunk_uux_hel(prec, sp, p->mp, g->d_edges, first_event + done, m, g->chunk, g->d_records, seed,
                                     iter, k > 0, g->d_partials, g->d_counters, w, grid, s, evk, g->d_hel_T, hsq)
              : launch_chunk_hel(p->ng, prec, sp, p->mp, g->d_edges, first_event + done, m, g->chunk, g->d_records,
                                 seed, iter, k > 0, g->d_partials, g->d_counters, w, grid, s, evk, g->d_hel_T, hsq);
      if (e != cudaSuccess) return cuda_fail(e, "mf_vegas_accumulate (helicity-sampled chunk kernels)");
      g_launches.fetch_add(2);
      continue;
    }
    switch (proc_key(p)) {
      case kUuxKey: e = launch_chunk_uux(prec, sp, p->mp, g->d_edges, first_event + done, m, g->chunk, g->d_records, seed, iter, k > 0, g->d_partials, g->d_counters, w, grid, s, evk); break;
      case kEeKey: e = launch_chunk_ee(prec, sp, p->mp, g->d_edges, first_event + done, m, g->chunk, g->d_records, seed, iter, k > 0, g->d_partials, g->d_counters, w, grid, s, evk); break;
      case 2: e = launch_chunk<2>(prec, sp, p->mp, g->d_edges, first_event + done, m, g->chunk, g->d_records, seed, iter, k > 0, g->d_partials, g->d_counters, w, grid, s, evk); break;
      case 3: e = launch_chunk<3>(prec, sp, p->mp, g->d_edges, first_event + done, m, g->chunk, g->d_records, seed, iter, k > 0, g->d_partials, g->d_counters, w, grid, s, evk); break;
      default: e = launch_chunk<4>(prec, sp, p->mp, g->d_edges, first_event + done, m, g->chunk, g->d_records, seed, iter, k > 0, g->d_partials, g->d_counters, w, grid, s, evk, p->me_warps); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "mf_vegas_accumulate (chunk kernels)");
    g_launches.fetch_add(2);
  }
  MF_CUDA(launch_reduce(g->d_partials, g->d_counters, grid, g->ndim, g->nbins, g->d_totals, s),
          "mf_vegas_accumulate (reduce)");
  g_launches.fetch_add(1);
  if (p->hel == 2) {
    MF_CUDA(launch_hel_reduce(g->d_hel_part, grid, g->hel_n, g->d_totals + 2 + g->ndim * g->nbins + 2, s),
            "mf_vegas_accumulate (helicity sums)");
    g_launches.fetch_add(1);
  }
  return MF_OK;
}

mf_status mf_grid_profile(mf_grid* g, int enable) {
  if (g == nullptr) return fail(MF_ERR_ARG, "mf_grid_profile: null argument");
  g->profile = enable != 0;
  g->ev_used = 0;
  return MF_OK;
}

mf_status mf_grid_profile_read(mf_grid* g, double* sample_ms, double* me_ms, int* chunks) {
  if (g == nullptr || sample_ms == nullptr || me_ms == nullptr || chunks == nullptr)
    return fail(MF_ERR_ARG, "mf_grid_profile_read: null argument");
  *sample_ms = *me_ms = 0.0;
  *chunks = g->ev_used / 3;
  if (g->ev_used == 0) return MF_OK;
  MF_CUDA(cudaEventSynchronize(g->ev[g->ev_used - 1]), "mf_grid_profile_read");
  for (int k = 0; k < g->ev_used / 3; ++k) {
    float a = 0, b = 0;
    MF_CUDA(cudaEventElapsedTime(&a, g->ev[3 * k], g->ev[3 * k + 1]), "mf_grid_profile_read");
    MF_CUDA(cudaEventElapsedTime(&b, g->ev[3 * k + 1], g->ev[3 * k + 2]), "mf_grid_profile_read");
    *sample_ms += a;
    *me_ms += b;
  }
  return MF_OK;
}

mf_status mf_grid_totals(mf_grid* g, double** totals, int* count) {
  if (g == nullptr || totals == nullptr || count == nullptr) return fail(MF_ERR_ARG, "mf_grid_totals: null argument");
  *totals = g->d_totals;
  *count = 2 + g->ndim * g->nbins + 2 + (g->proc->hel == 2 ? g->hel_n : 0);
  return MF_OK;
}

mf_status mf_grid_helicity(const mf_grid* g, double* prob, int n) {
  if (g == nullptr || prob == nullptr) return fail(MF_ERR_ARG, "mf_grid_helicity: null argument");
  if (g->hel_n == 0) return fail(MF_ERR_UNSUPPORTED, "mf_grid_helicity: the process has no helicity table");
  if (n != g->hel_n) return fail(MF_ERR_ARG, "mf_grid_helicity: n must be " + std::to_string(g->hel_n));
  std::vector<unsigned long long> T(n + 1);
  MF_CUDA(cudaMemcpy(T.data(), g->d_hel_T, sizeof(unsigned long long) * T.size(), cudaMemcpyDeviceToHost),
          "mf_grid_helicity");
  for (int h = 0; h < n; ++h) prob[h] = double(T[h + 1] - T[h]) * 2.3283064365386963e-10;   // 2^-32
  return MF_OK;
}

mf_status mf_grid_set_helicity(mf_grid* g, const double* prob, int n) {
  if (g == nullptr || prob == nullptr) return fail(MF_ERR_ARG, "mf_grid_set_helicity: null argument");
  if (g->hel_n == 0) return fail(MF_ERR_UNSUPPORTED, "mf_grid_set_helicity: the process has no helicity table");
  if (n != g->hel_n) return fail(MF_ERR_ARG, "mf_grid_set_helicity: n must be " + std::to_string(g->hel_n));
  double sum = 0.0;
  for (int h = 0; h < n; ++h) {
    if (!(prob[h] > 0.0) || !std::isfinite(prob[h]))
      return fail(MF_ERR_ARG, "mf_grid_set_helicity: every probability must be finite and > 0");
    sum += prob[h];
  }
  if (std::fabs(sum - 1.0) > 1e-9) return fail(MF_ERR_ARG, "mf_grid_set_helicity: the probabilities must sum to 1");
  std::vector<unsigned long long> T(n + 1);
  hel_thresholds(prob, n, T.data());
  for (int h = 0; h < n; ++h)
    if (T[h + 1] <= T[h])
      return fail(MF_ERR_ARG, "mf_grid_set_helicity: a probability below 2^-32 leaves its configuration undrawn");
  MF_CUDA(cudaMemcpy(g->d_hel_T, T.data(), sizeof(unsigned long long) * T.size(), cudaMemcpyHostToDevice),
          "mf_grid_set_helicity");
  return MF_OK;
}

mf_status mf_vegas_finish(mf_process* p, mf_grid* g, int64_t n_total, int refine, mf_result* out, void* stream) {
  if (p == nullptr || g == nullptr || out == nullptr) return fail(MF_ERR_ARG, "mf_vegas_finish: null argument");
  if (g->proc != p) return fail(MF_ERR_ARG, "mf_vegas_finish: grid belongs to another process");
  if (n_total < 2) return fail(MF_ERR_ARG, "mf_vegas_finish: need at least 2 events");
  if (refine < 0 || refine > 3) return fail(MF_ERR_ARG, "mf_vegas_finish: refine is a mask of 1 (edges) and 2 (helicity table)");
  cudaStream_t s = (cudaStream_t)stream;
  MF_CUDA(launch_finish(g->d_totals, g->ndim, g->nbins, n_total, refine & 1, g->d_edges, g->d_result, s),
          "mf_vegas_finish (estimate)");
  g_launches.fetch_add(1);
  if ((refine & 2) && p->hel == 2) {
    MF_CUDA(launch_hel_refine(g->d_totals + 2 + g->ndim * g->nbins + 2, g->hel_n, g->d_hel_T, s),
            "mf_vegas_finish (helicity table)");
    g_launches.fetch_add(1);
  }
  MF_CUDA(cudaMemcpyAsync(g->h_result, g->d_result, sizeof(double) * 6, cudaMemcpyDeviceToHost, s), "mf_vegas_finish (copy)");
  MF_CUDA(cudaStreamSynchronize(s), "mf_vegas_finish (sync)");
  return record_iteration(g, g->h_result, n_total, out);
}

mf_status mf_vegas_iterate(mf_process* p, mf_grid* g, uint64_t seed, int iter, int64_t n, int refine, mf_result* out,
                           double* weights, void* stream) {
  if (p == nullptr || g == nullptr || out == nullptr) return fail(MF_ERR_ARG, "mf_vegas_iterate: null argument");
  if (n < 2) return fail(MF_ERR_ARG, "mf_vegas_iterate: need at least 2 events");
  mf_status st = mf_vegas_accumulate(p, g, seed, iter, 0, n, weights, stream);
  if (st < 0) return st;
  return mf_vegas_finish(p, g, n, refine, out, stream);
}

mf_status mf_unweight(mf_process* p, mf_grid* g, uint64_t seed, int iter, int64_t first_event, int64_t n,
                      double w_max, int64_t capacity, double* momenta, double* weight, int64_t* event,
                      int64_t* n_kept, int64_t* n_over, void* stream) {
  if (p == nullptr || g == nullptr || n_kept == nullptr || n_over == nullptr)
    return fail(MF_ERR_ARG, "mf_unweight: null argument");
  if (g->proc != p) return fail(MF_ERR_ARG, "mf_unweight: grid belongs to another process");
  if (n < 1 || first_event < 0 || capacity < 0) return fail(MF_ERR_ARG, "mf_unweight: need n >= 1, first_event >= 0, capacity >= 0");
  if (!(w_max > 0) || !std::isfinite(w_max)) return fail(MF_ERR_ARG, "mf_unweight: w_max must be finite and > 0");
  if (capacity > 0 && (momenta == nullptr || weight == nullptr || event == nullptr))
    return fail(MF_ERR_ARG, "mf_unweight: null output buffer");
  cudaStream_t s = (cudaStream_t)stream;
  SampleParams sp = p->sp;
  sp.nbins = g->nbins;
  const int prec = p->precision == MF_FP64 ? 0 : 1;
  int acc_ctas = g->acc_ctas;
  if (p->hel) {
    const mf_status st = hel_grid_ctas(p, g);
    if (st != MF_OK) return st;
    acc_ctas = g->hel_ctas;
  }
  const int64_t cap = int64_t(p->sms) * effective_ctas(p, acc_ctas);
  MF_CUDA(cudaMemsetAsync(g->d_ucount, 0, 2 * sizeof(unsigned long long), s), "mf_unweight (counts)");
  for (int64_t done = 0; done < n; done += g->chunk) {
    const int64_t m = std::min(g->chunk, n - done);
    const int64_t ctas_needed = ((m + 31) / 32 + kWarps - 1) / kWarps;
    const int grid = int(std::min(std::min(cap, std::max<int64_t>(ctas_needed, 1)), int64_t(g->max_blocks)));
    // the chunk's weights: the iteration's kernels (their Vegas sums are not recorded)
    cudaError_t e;
    if (p->hel) {
      e = p->kind == 1
              ? launch_chunk_uux_hel(prec, sp, p->mp, g->d_edges, first_event + done, m, g->chunk, g->d_records, seed,
                                     iter, 0, g->d_partials, g->d_counters, g->d_wchunk, grid, s, nullptr, g->d_hel_T,
                                     nullptr)
              : launch_chunk_hel(p->ng, prec, sp, p->mp, g->d_edges, first_event + done, m, g->chunk, g->d_records,
                                 seed, iter, 0, g->d_partials, g->d_counters, g->d_wchunk, grid, s, nullptr,
                                 g->d_hel_T, nullptr);
    } else switch (proc_key(p)) {
      case kUuxKey: e = launch_chunk_uux(prec, sp, p->mp, g->d_edges, first_event + done, m, g->chunk, g->d_records, seed, iter, 0, g->d_partials, g->d_counters, g->d_wchunk, grid, s, nullptr); break;
      case kEeKey: e = launch_chunk_ee(prec, sp, p->mp, g->d_edges, first_event + done, m, g->chunk, g->d_records, seed, iter, 0, g->d_partials, g->d_counters, g->d_wchunk, grid, s, nullptr); break;
      case 2: e = launch_chunk<2>(prec, sp, p->mp, g->d_edges, first_event + done, m, g->chunk, g->d_records, seed, iter, 0, g->d_partials, g->d_counters, g->d_wchunk, grid, s); break;
      case 3: e = launch_chunk<3>(prec, sp, p->mp, g->d_edges, first_event + done, m, g->chunk, g->d_records, seed, iter, 0, g->d_partials, g->d_counters, g->d_wchunk, grid, s); break;
      default: e = launch_chunk<4>(prec, sp, p->mp, g->d_edges, first_event + done, m, g->chunk, g->d_records, seed, iter, 0, g->d_partials, g->d_counters, g->d_wchunk, grid, s, nullptr, p->me_warps); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "mf_unweight (chunk kernels)");
    MF_CUDA(launch_unweight(prec, g->d_records, sp.n_final, g->ndim, g->chunk, g->d_wchunk, m, seed, iter,
                            first_event + done, w_max, capacity, momenta, weight, event, g->d_ucount, s),
            "mf_unweight (hit or miss)");
    g_launches.fetch_add(3);
  }
  unsigned long long h[2] = {0, 0};
  MF_CUDA(cudaMemcpyAsync(h, g->d_ucount, sizeof(h), cudaMemcpyDeviceToHost, s), "mf_unweight (counts)");
  MF_CUDA(cudaStreamSynchronize(s), "mf_unweight (sync)");
  *n_kept = int64_t(h[0]);
  *n_over = int64_t(h[1]);
  return *n_kept > capacity ? MF_WARN_CAPACITY : MF_OK;
}

mf_status mf_fma_throughput(int precision, double* tflops) {
  if (tflops == nullptr || (precision != MF_FP64 && precision != MF_FP32)) return fail(MF_ERR_ARG, "mf_fma_throughput: bad argument");
  int dev = 0, sms = 0;
  MF_CUDA(cudaGetDevice(&dev), "mf_fma_throughput");
  MF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "mf_fma_throughput");
  float* sink = nullptr;
  MF_CUDA(cudaMalloc(&sink, sizeof(float) * sms * 64), "mf_fma_throughput");
  const int blocks = sms * 8;
  const int prec = precision == MF_FP64 ? 0 : 1;
  const int iters = precision == MF_FP64 ? 256 : 8192;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaError_t e = launch_fma_peak(prec, blocks, iters / 8, sink, 0);   // warm-up
  float ms = 0;
  if (e == cudaSuccess) {
    cudaEventRecord(a, 0);
    e = launch_fma_peak(prec, blocks, iters, sink, 0);
    cudaEventRecord(b, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "mf_fma_throughput");
  g_launches.fetch_add(2);
  const double flops = 2.0 * 8 * 16 * double(iters) * 256.0 * blocks;
  *tflops = flops / (double(ms) * 1e-3) / 1e12;
  return MF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of mf_vegas_accumulate.
//
// The fused kernel needs device scratch for its per-CTA partial sums.  Every
// other entry point takes it from buffers that mf_grid_create allocated.  Some
// host programs cannot allow that: a framework that carves all device memory
// out of its own arena up front and forbids the libraries it loads from
// calling cudaMalloc, or a process whose device-memory budget is already spent
// by the time it integrates.  For them the scratch below is a fixed array in
// the library's own device image, reserved when the library is loaded on a
// device and held there until the process exits.
//
// Limit: kStaticScratchBytes (2 MiB).  A CTA needs 2 + ndim*nbins doubles and
// two counters (at most 5.1 KB at 10 dimensions x 64 bins); the launch uses
// as many persistent CTAs as the occupancy allows and the array holds
// (at least 400 at the largest set-up), and strides over the events.
static constexpr size_t kStaticScratchBytes = size_t(2) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
unsigned char* g_static_ptr[kMaxDevices] = {nullptr};

// Device address of g_static_scratch on the current device.  Host code only
// holds a host-side stand-in for the symbol, so the address is looked up once
// per device (with that device current) and cached.
cudaError_t static_scratch(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (g_static_ptr[dev] == nullptr) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" mf_status mf_vegas_accumulate_static(mf_process* p, const double* edges, int nbins, uint64_t seed,
                                                 int iter, int64_t first_event, int64_t n, double* totals,
                                                 double* weights, void* stream) {
  if (p == nullptr || edges == nullptr || totals == nullptr)
    return fail(MF_ERR_ARG, "mf_vegas_accumulate_static: null argument");
  if (p->kind != 0)
    return fail(MF_ERR_UNSUPPORTED, "mf_vegas_accumulate_static: covers the gluon-initiated processes");
  if (p->hel)
    return fail(MF_ERR_UNSUPPORTED, "mf_vegas_accumulate_static: sums the helicities (helicity sampling is on)");
  if (nbins < 2 || nbins > 64) return fail(MF_ERR_ARG, "mf_vegas_accumulate_static: nbins must be in [2, 64]");
  if (n < 1 || first_event < 0) return fail(MF_ERR_ARG, "mf_vegas_accumulate_static: need n >= 1 and first_event >= 0");
  size_t smem = 0;
  int ctas = 0;
  cudaError_t e = dispatch_fused_config(p->ng, p->precision, p->ndim, nbins, &smem, &ctas);
  if (e != cudaSuccess) return cuda_fail(e, "mf_vegas_accumulate_static (configuration)");
  if (ctas < 1)
    return fail(MF_ERR_UNSUPPORTED, "mf_vegas_accumulate_static: the fused kernel's shared memory (" +
                                        std::to_string(smem) + " bytes) does not fit on an SM");
  // per-CTA scratch: the CTA's partial sums, then (after all CTAs' sums) its
  // two counters; the grid shrinks to what the reserved array holds (the
  // kernel strides over the events, so the result does not depend on it)
  const size_t nacc = 2 + size_t(p->ndim) * nbins;
  const size_t per_cta = sizeof(double) * nacc + sizeof(unsigned long long) * 2;
  const int64_t fit = int64_t((kStaticScratchBytes - 256) / per_cta);
  if (fit < 1)
    return fail(MF_ERR_ARG, "mf_vegas_accumulate_static: one CTA needs " + std::to_string(per_cta + 256) +
                                " bytes of scratch, more than the " + std::to_string(kStaticScratchBytes) +
                                " bytes reserved in the library");
  const int64_t ntiles = (n + kTile - 1) / kTile;
  int64_t cap = int64_t(p->sms) * effective_ctas(p, ctas);
  if (cap > fit) cap = fit;
  const int grid = int(ntiles < cap ? ntiles : cap);
  const size_t part_bytes = sizeof(double) * nacc * size_t(grid);
  const size_t cnt_off = (part_bytes + 255) & ~size_t(255);
  unsigned char* scratch = nullptr;
  e = static_scratch(&scratch);
  if (e != cudaSuccess) return cuda_fail(e, "mf_vegas_accumulate_static (scratch address)");
  double* partials = reinterpret_cast<double*>(scratch);
  unsigned long long* counters = reinterpret_cast<unsigned long long*>(scratch + cnt_off);
  cudaStream_t s = (cudaStream_t)stream;
  SampleParams sp = p->sp;
  sp.nbins = nbins;
  const int prec = p->precision == MF_FP64 ? 0 : 1;
  switch (p->ng) {
    case 2: e = launch_fused<2>(prec, sp, p->mp, edges, first_event, n, seed, iter, partials, counters, weights, grid, s); break;
    case 3: e = launch_fused<3>(prec, sp, p->mp, edges, first_event, n, seed, iter, partials, counters, weights, grid, s); break;
    default: e = launch_fused<4>(prec, sp, p->mp, edges, first_event, n, seed, iter, partials, counters, weights, grid, s); break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "mf_vegas_accumulate_static (fused kernel)");
  g_launches.fetch_add(1);
  e = launch_reduce(partials, counters, grid, p->ndim, nbins, totals, s);
  if (e != cudaSuccess) return cuda_fail(e, "mf_vegas_accumulate_static (reduce)");
  g_launches.fetch_add(1);
  return MF_OK;
}

