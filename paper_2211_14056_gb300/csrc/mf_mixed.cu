// Several processes in one iteration (the batched mixed launch;
// arXiv:2211.14056 Sec. 3, Fig. 3: how the work is spread over blocks and
// threads decides the run time, so the launch shape is tuned, not fixed).
//
//   k_sample_mixed : one launch samples every process's events (thread per
//                    event) into per-process records and pass lists;
//   k_me_mixed     : one persistent launch; warps take tiles of listed events
//                    from a single work queue ordered by cost (the 2->4
//                    process first), so the expensive tiles start early and
//                    the cheap ones fill the tail; per-process Vegas sums;
//   then the per-process deterministic reduction and refinement.
// A plan (mf_mixed) owns the queue, the iteration counter and an optional
// CUDA graph of the whole iteration, replayed with a new iteration number.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "mf_internal.h"

namespace mf {

constexpr int kMaxProc = 8;

template <typename K> struct MixedArgs {
  int nproc;
  int ng[kMaxProc];             // gluon count; 0 for u u~ -> t t~ g g (not in the shared queue)
  int ndim[kMaxProc], nbins[kMaxProc];
  int64_t n[kMaxProc];          // events of each process
  int64_t off[kMaxProc + 1];    // prefix sums of n
  SampleParams sp[kMaxProc];
  MeParams mp[kMaxProc];
  const double* edges[kMaxProc];
  RecordView<K> rec[kMaxProc];
  double* partials[kMaxProc];
  unsigned long long* counters[kMaxProc];
  double* w_out[kMaxProc];
  unsigned* queue;              // work-queue head (zero on entry)
  const unsigned* iter_seed;    // [0] iteration, [1] seed low, [2] seed high (device)
  int tile;                     // listed events per work item
};

template <typename K>
__global__ void __launch_bounds__(kThreads) k_sample_mixed(MixedArgs<K> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* edges = reinterpret_cast<double*>(smem_raw);
  int eoff[kMaxProc + 1];
  eoff[0] = 0;
  for (int p = 0; p < a.nproc; ++p) eoff[p + 1] = eoff[p] + a.ndim[p] * (a.nbins[p] + 1);
  for (int p = 0; p < a.nproc; ++p)
    for (int i = threadIdx.x; i < a.ndim[p] * (a.nbins[p] + 1); i += blockDim.x) edges[eoff[p] + i] = a.edges[p][i];
  __syncthreads();
  const int iter = int(a.iter_seed[0]);
  const uint64_t seed = uint64_t(a.iter_seed[1]) | (uint64_t(a.iter_seed[2]) << 32);
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  const int64_t total = a.off[a.nproc];
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < total; base += stride) {
    const int64_t g = base + threadIdx.x;
    int p = 0;
    while (p + 1 < a.nproc && g >= a.off[p + 1]) ++p;
    const int64_t e = g - a.off[p];
    int pass = 0, fail = 0;
    if (g < total) {
      EventKin<K> k;
      sample_event(a.sp[p], edges + eoff[p], seed, iter, uint64_t(e), k);
      const RecordView<K>& r = a.rec[p];
#pragma unroll
      for (int i = 0; i < kMaxExt - 2; ++i)
        if (i < a.sp[p].n_final)
#pragma unroll
          for (int c = 0; c < 4; ++c) r.mom[int64_t(i * 4 + c) * r.C + e] = k.p[2 + i][c];
      r.rs[e] = k.p[0][0] + k.p[1][0];
      r.pref[e] = k.prefactor;
#pragma unroll
      for (int j = 0; j < kMaxDim; ++j)
        if (j < a.ndim[p]) r.flag[int64_t(j) * r.C + e] = k.bins[j];
      pass = k.pass;
      fail = k.newton_fail;
      if (!pass && a.w_out[p] != nullptr) a.w_out[p][e] = 0.0;
    }
    // compaction per process: lanes of a warp may belong to two processes at a boundary
    for (int q = 0; q < a.nproc; ++q) {
      const bool mine = (g < total) && (p == q);
      const unsigned bal = __ballot_sync(full, mine && pass);
      const unsigned fbal = __ballot_sync(full, mine && fail);
      if (!bal && !fbal) continue;
      unsigned pos = 0;
      if (lane == 0) {
        if (bal) pos = atomicAdd(&a.rec[q].count[0], unsigned(__popc(bal)));
        if (fbal) atomicAdd(&a.rec[q].count[1], unsigned(__popc(fbal)));
      }
      pos = __shfl_sync(full, pos, 0);
      if (mine && pass) a.rec[q].list[pos + __popc(bal & ((1u << lane) - 1u))] = int(e);
    }
  }
}

template <typename T> struct MixedLayout {
  __host__ __device__ static size_t al(size_t x) { return (x + 15) & ~size_t(15); }
  // per-process accumulators: [sum w, sum w^2, hist]
  __host__ __device__ static size_t acc_bytes(const int* ndim, const int* nbins, int nproc) {
    size_t b = 0;
    for (int p = 0; p < nproc; ++p) b += sizeof(double) * (2 + ndim[p] * nbins[p]);
    return al(b);
  }
  __host__ __device__ static size_t total(const int* ndim, const int* nbins, int nproc) {
    return acc_bytes(ndim, nbins, nproc) + WarpMem<4, T>::bytes * kWarps;
  }
};

// One tile of listed events of process p on this warp.
template <int NG, typename T>
__device__ __forceinline__ void mixed_tile(const MixedArgs<T>& a, int p, int64_t first, int64_t last,
                                           unsigned char* wm, double* acc, double& s1, double& s2) {
  constexpr int EPW = Lanes<NG>::EPW, L = Lanes<NG>::L, NEXT = Lanes<NG>::NEXT;
  const int lane = threadIdx.x & 31, group = lane / L, gl = lane % L;
  const RecordView<T>& r = a.rec[p];
  const MeParams& mp = a.mp[p];
  const T mt = T(mp.mt), mw = T(mp.mw);
  const int nbins = a.nbins[p], ndim = a.ndim[p];
  for (int64_t base = first; base < last; base += EPW) {
    const int64_t k = base + group;
    const bool ok = k < last;
    const int64_t e = r.list[ok ? k : base];
    T pp[NEXT][4];
    const T rs = r.rs[e];
    pp[0][0] = T(0.5) * rs; pp[0][1] = T(0); pp[0][2] = T(0); pp[0][3] = T(0.5) * rs;
    pp[1][0] = T(0.5) * rs; pp[1][1] = T(0); pp[1][2] = T(0); pp[1][3] = T(-0.5) * rs;
#pragma unroll
    for (int i = 0; i < NG; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) pp[2 + i][c] = r.mom[int64_t(i * 4 + c) * r.C + e];
    const T v = group_me2<NG, T>(pp, wm, group, gl, mt, mw, mp.colour_tc);
    if (ok) {
      const double w = double(v) * mp.norm * r.pref[e];
      if (gl == 0) {
        s1 += w;
        s2 += w * w;
        if (a.w_out[p] != nullptr) a.w_out[p][e] = w;
      }
      if (gl < ndim) atomicAdd(&acc[2 + gl * nbins + r.flag[int64_t(gl) * r.C + e]], w * w);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 2) k_me_mixed(MixedArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int64_t tiles_off[kMaxProc + 1];
  __shared__ unsigned item_s[kWarps];
  double* acc = reinterpret_cast<double*>(smem_raw);
  int aoff[kMaxProc + 1];
  aoff[0] = 0;
  for (int p = 0; p < a.nproc; ++p) aoff[p + 1] = aoff[p] + 2 + a.ndim[p] * a.nbins[p];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  unsigned char* wm = smem_raw + MixedLayout<T>::acc_bytes(a.ndim, a.nbins, a.nproc) + warp * WarpMem<4, T>::bytes;
  for (int i = t; i < aoff[a.nproc]; i += kThreads) acc[i] = 0.0;
  if (t == 0) {
    tiles_off[0] = 0;
    for (int p = 0; p < a.nproc; ++p) {
      const int64_t np = a.ng[p] == 0 ? 0 : a.rec[p].count[0];
      tiles_off[p + 1] = tiles_off[p] + (np + a.tile - 1) / a.tile;
    }
  }
  __syncthreads();
  const int64_t total = tiles_off[a.nproc];
  double s1[kMaxProc] = {0.0, 0.0, 0.0, 0.0}, s2[kMaxProc] = {0.0, 0.0, 0.0, 0.0};
  while (true) {
    if (lane == 0) item_s[warp] = atomicAdd(a.queue, 1u);
    __syncwarp();
    const int64_t item = item_s[warp];
    __syncwarp();
    if (item >= total) break;
    int p = 0;
    while (p + 1 < a.nproc && item >= tiles_off[p + 1]) ++p;
    const int64_t tl = item - tiles_off[p];
    const int64_t np = a.rec[p].count[0];
    const int64_t first = tl * a.tile;
    const int64_t last = (first + a.tile < np) ? first + a.tile : np;
    double x1 = 0.0, x2 = 0.0;
    switch (a.ng[p]) {
      case 2: mixed_tile<2, T>(a, p, first, last, wm, acc + aoff[p], x1, x2); break;
      case 3: mixed_tile<3, T>(a, p, first, last, wm, acc + aoff[p], x1, x2); break;
      default: mixed_tile<4, T>(a, p, first, last, wm, acc + aoff[p], x1, x2); break;
    }
    for (int q = 0; q < kMaxProc; ++q)
      if (q == p) { s1[q] += x1; s2[q] += x2; }
  }
  const unsigned full = 0xffffffffu;
  for (int p = 0; p < a.nproc; ++p) {
    double x1 = s1[p], x2 = s2[p];
    for (int off = 16; off > 0; off >>= 1) {
      x1 += __shfl_xor_sync(full, x1, off);
      x2 += __shfl_xor_sync(full, x2, off);
    }
    if (lane == 0) {
      atomicAdd(&acc[aoff[p]], x1);
      atomicAdd(&acc[aoff[p] + 1], x2);
    }
  }
  __syncthreads();
  for (int p = 0; p < a.nproc; ++p) {
    const int nacc = 2 + a.ndim[p] * a.nbins[p];
    double* dst = a.partials[p] + int64_t(blockIdx.x) * nacc;
    for (int i = t; i < nacc; i += kThreads) dst[i] = acc[aoff[p] + i];
    if (t < 2)
      a.counters[p][blockIdx.x * 2 + t] =
          (blockIdx.x == 0 && a.ng[p] != 0) ? (unsigned long long)a.rec[p].count[t] : 0ull;
  }
}

}  // namespace mf

using namespace mf;
using namespace mf::detail;

struct mf_mixed {
  int nproc = 0;
  int precision = 0;                 // 0 FP64, 1 FP32 (every process the same)
  mf_process* procs[kMaxProc] = {};
  mf_grid* grids[kMaxProc] = {};
  int64_t n[kMaxProc] = {};
  int order[kMaxProc] = {};          // processes by decreasing cost (gluon count)
  int ctas_per_sm = 0;               // 0 = occupancy
  int occupancy = 1;
  int tile = 32;                     // listed events per work item; 0: per-process kernels
  bool queue_fits = true;            // the shared-queue kernel fits on an SM (its shared memory holds
                                     // every process's sums beside the warps' 2->4 stores)
  int acc_occ[kMaxProc] = {};        // occupancy of each process's own |M|^2 kernel
  size_t me_smem = 0, sample_smem = 0;
  unsigned* d_queue = nullptr;
  unsigned* d_iter = nullptr;        // [iteration, seed lo, seed hi]
  unsigned* h_iter = nullptr;        // pinned
  int sms = 0;
  bool use_graph = false;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};   // refine off / on
  cudaStream_t captured_on[2] = {nullptr, nullptr};
};

namespace {

int me_grid(const mf_mixed* m) {
  const int c = m->ctas_per_sm > 0 && m->ctas_per_sm < m->occupancy ? m->ctas_per_sm : m->occupancy;
  return m->sms * (c < 1 ? 1 : c);
}

// CTAs of process k's own |M|^2 kernel (per-process mode)
int acc_grid(const mf_mixed* m, int k) {
  const int occ = m->acc_occ[k];
  const int c = m->ctas_per_sm > 0 && m->ctas_per_sm < occ ? m->ctas_per_sm : occ;
  return m->sms * (c < 1 ? 1 : c);
}

cudaError_t launch_acc_dispatch(int key, int prec, const MeParams& mp, int n_final, int ndim, int nbins, void* rec,
                                int64_t C, int accumulate, double* partials, unsigned long long* counters, int grid,
                                cudaStream_t s) {
  if (key == kUuxKey)
    return launch_me_acc_uux(prec, mp, n_final, ndim, nbins, rec, C, accumulate, partials, counters, nullptr, grid, s);
  if (key == kEeKey)
    return launch_me_acc_ee(prec, mp, n_final, ndim, nbins, rec, C, accumulate, partials, counters, nullptr, grid, s);
  switch (key) {
    case 2: return launch_me_acc<2>(prec, mp, n_final, ndim, nbins, rec, C, accumulate, partials, counters, nullptr, grid, s);
    case 3: return launch_me_acc<3>(prec, mp, n_final, ndim, nbins, rec, C, accumulate, partials, counters, nullptr, grid, s);
    default: return launch_me_acc<4>(prec, mp, n_final, ndim, nbins, rec, C, accumulate, partials, counters, nullptr, grid, s);
  }
}

template <typename K>
MixedArgs<K> make_args(const mf_mixed* m) {
  MixedArgs<K> a;
  std::memset(&a, 0, sizeof(a));
  a.nproc = m->nproc;
  a.off[0] = 0;
  for (int k = 0; k < m->nproc; ++k) {
    const int i = m->order[k];
    const mf_process* p = m->procs[i];
    const mf_grid* g = m->grids[i];
    a.ng[k] = p->kind == 0 ? p->ng : 0;
    a.ndim[k] = g->ndim;
    a.nbins[k] = g->nbins;
    a.n[k] = m->n[i];
    a.off[k + 1] = a.off[k] + m->n[i];
    a.sp[k] = p->sp;
    a.sp[k].nbins = g->nbins;
    a.mp[k] = p->mp;
    a.edges[k] = g->d_edges;
    a.rec[k] = RecordView<K>::carve(g->d_records, p->sp.n_final, g->ndim, g->chunk);
    a.partials[k] = g->d_partials;
    a.counters[k] = g->d_counters;
    a.w_out[k] = nullptr;
  }
  a.queue = m->d_queue;
  a.iter_seed = m->d_iter;
  a.tile = m->tile;
  return a;
}

// enqueue one mixed iteration on s (capturable: no allocation, no host sync)
mf_status enqueue(mf_mixed* m, int refine, cudaStream_t s) {
  MF_CUDA(cudaMemcpyAsync(m->d_iter, m->h_iter, 3 * sizeof(unsigned), cudaMemcpyHostToDevice, s), "mf_mixed (iteration)");
  for (int k = 0; k < m->nproc; ++k) {
    const mf_grid* g = m->grids[m->order[k]];
    const mf_process* p = m->procs[m->order[k]];
    unsigned* cnt = (m->precision == 0)
                        ? RecordView<double>::carve(g->d_records, p->sp.n_final, g->ndim, g->chunk).count
                        : RecordView<float>::carve(g->d_records, p->sp.n_final, g->ndim, g->chunk).count;
    MF_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned), s), "mf_mixed (counts)");
  }
  MF_CUDA(cudaMemsetAsync(m->d_queue, 0, sizeof(unsigned), s), "mf_mixed (queue)");
  int64_t total = 0;
  for (int k = 0; k < m->nproc; ++k) total += m->n[k];
  const int64_t need = (total + kThreads - 1) / kThreads;
  const int sgrid = int(need < int64_t(m->sms) * 16 ? need : int64_t(m->sms) * 16);
  const int grid = me_grid(m);
  const bool queue = m->tile > 0;
  if (m->precision == 0) {
    const MixedArgs<double> a = make_args<double>(m);
    k_sample_mixed<double><<<sgrid, kThreads, m->sample_smem, s>>>(a);
    if (queue) k_me_mixed<double><<<grid, kThreads, m->me_smem, s>>>(a);
  } else {
    const MixedArgs<float> a = make_args<float>(m);
    k_sample_mixed<float><<<sgrid, kThreads, m->sample_smem, s>>>(a);
    if (queue) k_me_mixed<float><<<grid, kThreads, m->me_smem, s>>>(a);
  }
  MF_CUDA(cudaGetLastError(), "mf_mixed (kernels)");
  count_launches(queue ? 2 : 1);
  if (!queue) {
    // per-process mode: each process's own |M|^2 kernel, most expensive first
    for (int k = 0; k < m->nproc; ++k) {
      const int i = m->order[k];
      const mf_process* p = m->procs[i];
      mf_grid* g = m->grids[i];
      MF_CUDA(launch_acc_dispatch(proc_key(p), m->precision, p->mp, p->sp.n_final, g->ndim, g->nbins, g->d_records,
                                  g->chunk, 0, g->d_partials, g->d_counters, acc_grid(m, i), s),
              "mf_mixed (per-process kernel)");
      count_launches(1);
    }
  } else {
    // the shared queue covers the gluon-initiated processes; u u~ -> t t~ g g
    // and e+ e- -> mu+ mu- run their own kernels on the queue's CTA count,
    // adding to the partials the queue kernel zeroed
    for (int k = 0; k < m->nproc; ++k) {
      const mf_process* p = m->procs[k];
      if (p->kind == 0) continue;
      mf_grid* g = m->grids[k];
      MF_CUDA(launch_acc_dispatch(proc_key(p), m->precision, p->mp, p->sp.n_final, g->ndim, g->nbins, g->d_records,
                                  g->chunk, 1, g->d_partials, g->d_counters, grid, s),
              "mf_mixed (own kernel)");
      count_launches(1);
    }
  }
  for (int k = 0; k < m->nproc; ++k) {
    mf_grid* g = m->grids[k];
    const int pgrid = queue ? grid : acc_grid(m, k);
    MF_CUDA(launch_reduce(g->d_partials, g->d_counters, pgrid, g->ndim, g->nbins, g->d_totals, s), "mf_mixed (reduce)");
    MF_CUDA(launch_finish(g->d_totals, g->ndim, g->nbins, m->n[k], refine, g->d_edges, g->d_result, s), "mf_mixed (finish)");
    MF_CUDA(cudaMemcpyAsync(g->h_result, g->d_result, sizeof(double) * 6, cudaMemcpyDeviceToHost, s), "mf_mixed (copy)");
    count_launches(2);
  }
  return MF_OK;
}

void drop_graphs(mf_mixed* m) {
  for (int r = 0; r < 2; ++r) {
    if (m->exec[r]) cudaGraphExecDestroy(m->exec[r]);
    m->exec[r] = nullptr;
  }
}

}  // namespace

extern "C" {

mf_status mf_mixed_create(mf_process* const* procs, mf_grid* const* grids, const int64_t* n, int nproc,
                          mf_mixed** out) {
  if (procs == nullptr || grids == nullptr || n == nullptr || out == nullptr)
    return fail(MF_ERR_ARG, "mf_mixed_create: null argument");
  if (nproc < 1 || nproc > kMaxProc) return fail(MF_ERR_ARG, "mf_mixed_create: 1 to 8 processes");
  *out = nullptr;
  mf_mixed* m = new mf_mixed();
  m->nproc = nproc;
  for (int k = 0; k < nproc; ++k) {
    if (procs[k] == nullptr || grids[k] == nullptr || grids[k]->proc != procs[k] || n[k] < 2) {
      delete m;
      return fail(MF_ERR_ARG, "mf_mixed_create: process " + std::to_string(k) + ": bad process, grid or event count");
    }
    if (procs[k]->hel) {
      delete m;
      return fail(MF_ERR_UNSUPPORTED, "mf_mixed_create: process " + std::to_string(k) +
                                          " samples helicities; a mixed plan sums them");
    }
    const int prec = procs[k]->precision == MF_FP64 ? 0 : 1;
    if (k > 0 && prec != m->precision) {
      delete m;
      return fail(MF_ERR_ARG, "mf_mixed_create: every process must use the same precision");
    }
    if (n[k] > (int64_t(1) << 31) - 1) {
      delete m;
      return fail(MF_ERR_ARG, "mf_mixed_create: at most 2^31 - 1 events per process");
    }
    m->precision = prec;
    m->procs[k] = procs[k];
    m->grids[k] = grids[k];
    m->n[k] = n[k];
    m->order[k] = k;
  }
  std::stable_sort(m->order, m->order + nproc, [&](int a, int b) { return procs[a]->ng > procs[b]->ng; });
  m->sms = procs[0]->sms;
  // shared memory of both kernels
  int ndim[kMaxProc], nbins[kMaxProc];
  size_t esm = 0;
  for (int k = 0; k < nproc; ++k) {
    ndim[k] = grids[m->order[k]]->ndim;
    nbins[k] = grids[m->order[k]]->nbins;
    esm += sizeof(double) * ndim[k] * (nbins[k] + 1);
  }
  m->sample_smem = esm;
  cudaError_t e = cudaSuccess;
  int smem_optin = 0;
  e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, procs[0]->device);
  m->me_smem = m->precision == 0 ? MixedLayout<double>::total(ndim, nbins, nproc)
                                 : MixedLayout<float>::total(ndim, nbins, nproc);
  m->occupancy = 0;
  if (e == cudaSuccess && m->me_smem <= size_t(smem_optin)) {
    if (m->precision == 0) {
      e = cudaFuncSetAttribute(k_me_mixed<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(m->me_smem));
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m->occupancy, k_me_mixed<double>, kThreads, m->me_smem);
    } else {
      e = cudaFuncSetAttribute(k_me_mixed<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(m->me_smem));
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m->occupancy, k_me_mixed<float>, kThreads, m->me_smem);
    }
  }
  if (e == cudaSuccess && m->occupancy < 1) {
    // too many processes' sums for the shared queue: the plan runs the
    // per-process form only
    m->queue_fits = false;
    m->occupancy = 0;
    m->tile = 0;
  }
  for (int k = 0; k < nproc && e == cudaSuccess; ++k) {
    size_t asm_ = 0;
    e = dispatch_acc_config(proc_key(procs[k]), m->precision, grids[k]->ndim, grids[k]->nbins, &asm_, &m->acc_occ[k]);
    if (e == cudaSuccess && m->acc_occ[k] < 1) e = cudaErrorInvalidConfiguration;
  }
  // per-grid records for the whole event count, and partial slots for the mixed grid
  for (int k = 0; k < nproc && e == cudaSuccess; ++k) {
    mf_status st = grid_reserve(grids[k], n[k]);
    if (st != MF_OK) {
      delete m;
      return st;
    }
    if (grids[k]->max_blocks < m->sms * std::max(m->occupancy, m->acc_occ[k])) {
      delete m;
      return fail(MF_ERR_ARG, "mf_mixed_create: grid scratch smaller than the mixed launch");
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&m->d_queue, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_iter, 4 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMallocHost(&m->h_iter, 4 * sizeof(unsigned));
  if (e != cudaSuccess) {
    mf_mixed_destroy(m);
    return cuda_fail(e, "mf_mixed_create");
  }
  *out = m;
  return MF_OK;
}

mf_status mf_mixed_destroy(mf_mixed* m) {
  if (m == nullptr) return MF_OK;
  drop_graphs(m);
  cudaFree(m->d_queue);
  cudaFree(m->d_iter);
  cudaFreeHost(m->h_iter);
  delete m;
  return MF_OK;
}

mf_status mf_mixed_set_launch(mf_mixed* m, int ctas_per_sm, int tile) {
  if (m == nullptr || ctas_per_sm < 0 || tile < 0) return fail(MF_ERR_ARG, "mf_mixed_set_launch: bad argument");
  if (tile > 0 && !m->queue_fits)
    return fail(MF_ERR_UNSUPPORTED, "mf_mixed_set_launch: the shared-queue kernel does not fit on an SM for this "
                                    "plan (per-process form only, tile = 0)");
  m->ctas_per_sm = ctas_per_sm;
  m->tile = tile;
  drop_graphs(m);
  return MF_OK;
}

mf_status mf_mixed_use_graph(mf_mixed* m, int enable) {
  if (m == nullptr) return fail(MF_ERR_ARG, "mf_mixed_use_graph: null argument");
  m->use_graph = enable != 0;
  if (!m->use_graph) drop_graphs(m);
  return MF_OK;
}

mf_status mf_mixed_run(mf_mixed* m, uint64_t seed, int iter, int refine, mf_result* out, void* stream) {
  if (m == nullptr || out == nullptr) return fail(MF_ERR_ARG, "mf_mixed_run: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int r = refine ? 1 : 0;
  m->h_iter[0] = unsigned(iter);
  m->h_iter[1] = unsigned(seed);
  m->h_iter[2] = unsigned(seed >> 32);
  // the legacy default stream cannot be captured: run it directly there
  if (m->use_graph && s != nullptr) {
    if (m->exec[r] == nullptr || m->captured_on[r] != s) {
      if (m->exec[r]) cudaGraphExecDestroy(m->exec[r]);
      m->exec[r] = nullptr;
      cudaGraph_t graph = nullptr;
      MF_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "mf_mixed_run (capture)");
      mf_status st = enqueue(m, r, s);
      cudaError_t e = cudaStreamEndCapture(s, &graph);
      if (st != MF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(e, "mf_mixed_run (end capture)");
      e = cudaGraphInstantiate(&m->exec[r], graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(e, "mf_mixed_run (instantiate)");
      m->captured_on[r] = s;
    }
    MF_CUDA(cudaGraphLaunch(m->exec[r], s), "mf_mixed_run (graph launch)");
  } else {
    mf_status st = enqueue(m, r, s);
    if (st != MF_OK) return st;
  }
  MF_CUDA(cudaStreamSynchronize(s), "mf_mixed_run (sync)");
  mf_status worst = MF_OK;
  for (int k = 0; k < m->nproc; ++k) {
    mf_status st = record_iteration(m->grids[k], m->grids[k]->h_result, m->n[k], &out[k]);
    if (st < 0) return st;
    if (st > worst) worst = st;
  }
  return worst;
}

mf_status mf_mixed_autotune(mf_mixed* m, uint64_t seed, int ncand, const int* cand_ctas, const int* cand_tile,
                            double* ms, int* best, void* stream) {
  if (m == nullptr || ncand < 1 || cand_ctas == nullptr || cand_tile == nullptr || ms == nullptr || best == nullptr)
    return fail(MF_ERR_ARG, "mf_mixed_autotune: bad argument");
  for (int c = 0; c < ncand; ++c)
    if (cand_ctas[c] < 0 || cand_tile[c] < 0) return fail(MF_ERR_ARG, "mf_mixed_autotune: bad candidate");
  for (int c = 0; c < ncand; ++c)
    if (cand_tile[c] > 0 && !m->queue_fits)
      return fail(MF_ERR_UNSUPPORTED, "mf_mixed_autotune: a shared-queue candidate for a plan that runs the "
                                      "per-process form only");
  cudaStream_t s = (cudaStream_t)stream;
  const int keep_c = m->ctas_per_sm, keep_t = m->tile;
  const bool keep_g = m->use_graph;
  m->use_graph = false;
  cudaEvent_t a, b;
  MF_CUDA(cudaEventCreate(&a), "mf_mixed_autotune");
  MF_CUDA(cudaEventCreate(&b), "mf_mixed_autotune");
  // the grids must not drift while tuning: no refinement, results discarded
  std::vector<std::vector<double>> keepI(m->nproc), keepV(m->nproc);
  for (int k = 0; k < m->nproc; ++k) {
    keepI[k] = m->grids[k]->Ik;
    keepV[k] = m->grids[k]->vark;
  }
  *best = 0;
  mf_status st = MF_OK;
  for (int c = 0; c < ncand && st >= 0; ++c) {
    m->ctas_per_sm = cand_ctas[c];
    m->tile = cand_tile[c];
    m->h_iter[0] = 0;
    m->h_iter[1] = unsigned(seed);
    m->h_iter[2] = unsigned(seed >> 32);
    st = enqueue(m, 0, s);                      // warm-up
    if (st < 0) break;
    cudaEventRecord(a, s);
    st = enqueue(m, 0, s);
    cudaEventRecord(b, s);
    if (st < 0) break;
    cudaError_t e = cudaEventSynchronize(b);
    float t = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (e != cudaSuccess) { st = cuda_fail(e, "mf_mixed_autotune"); break; }
    ms[c] = t;
    if (t < ms[*best]) *best = c;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  for (int k = 0; k < m->nproc; ++k) {
    m->grids[k]->Ik = keepI[k];
    m->grids[k]->vark = keepV[k];
  }
  m->use_graph = keep_g;
  drop_graphs(m);
  if (st < 0) {
    m->ctas_per_sm = keep_c;
    m->tile = keep_t;
    return st;
  }
  m->ctas_per_sm = cand_ctas[*best];
  m->tile = cand_tile[*best];
  return MF_OK;
}

}  // extern "C"
