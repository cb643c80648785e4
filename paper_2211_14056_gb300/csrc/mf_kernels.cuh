// Kernels of the hot path for a top pair plus NG gluons (gg -> t tbar + (NG-2) g):
//   k_matrix_element : |M|^2 of given momenta (one lane group per event)
//   k_sample         : per-event kinematics only (one thread per event)
//   k_fused          : sample + |M|^2 + Vegas accumulation, persistent CTAs
//   k_reduce, k_finish (mf_kernels_common.cu): deterministic sum of the per-CTA
//                      partials, then estimate and grid refinement
//
// Work split of one event's |M|^2 over L = 2^(NG+1) lanes (arXiv:2211.14056,
// Sec. 2: the paper moves exactly this per-event matrix element into one
// device operator; here it is one lane group of one fused kernel):
//   lane bits 0..NG-1 = gluon helicities, bit NG = tbar helicity; every lane
//   sums both top helicities.  The colour-ordered gluon sub-currents G(B),
//   which only depend on the helicities of the gluons in B, are computed once
//   per event by the whole group and kept in shared memory; each lane then
//   runs the straight-line quark-line code of mf_gen_ttng.cuh and its own
//   colour sum, and the group reduces with xor shuffles.  No per-diagram
//   tensor leaves the SM (the memory-footprint point of Sec. 2).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mf_device.cuh"
#include "mf_gen_ttng.cuh"
#include "mf_sample.cuh"

namespace mf {

struct MeParams {
  double mt, mw;     // top mass, mass * width
  double norm;       // g^(2 NG) / (spin-colour average * identical-particle factor * colour denominator)
};

template <int NG> struct Lanes {
  static constexpr int L = 2 << NG;        // lanes per event
  static constexpr int EPW = 32 / L;       // events per warp
  static constexpr int NEXT = NG + 2;
};

template <int NG>
__device__ __forceinline__ unsigned pdep_mask(unsigned c, unsigned mask) {
  unsigned H = 0;
  int j = 0;
#pragma unroll
  for (int g = 0; g < NG; ++g)
    if (mask >> g & 1u) { H |= ((c >> j) & 1u) << g; ++j; }
  return H;
}

template <int NG>
__device__ __forceinline__ unsigned pext_mask(unsigned H, unsigned mask) {
  unsigned c = 0;
  int j = 0;
#pragma unroll
  for (int g = 0; g < NG; ++g)
    if (mask >> g & 1u) { c |= ((H >> g) & 1u) << j; ++j; }
  return c;
}

template <int NG, typename T>
__device__ __forceinline__ V4<T> load_block(const V4<T>* Gs, uint8_t ref, unsigned H) {
  const int id = ref & 0x7f;
  V4<T> g = Gs[blk_off<NG>()[id] + pext_mask<NG>(H, blk_mask<NG>()[id])];
  if (ref & 0x80) g = neg(g);
  return g;
}

template <int NG, typename T>
__device__ __forceinline__ R4<T> block_momentum(const R4<T>* q, unsigned mask) {
  R4<T> P = {{T(0), T(0), T(0), T(0)}};
#pragma unroll
  for (int g = 0; g < NG; ++g)
    if (mask >> g & 1u) P = P + q[g];
  return P;
}

// one level (block length K) of the colour-ordered gluon currents
template <int NG, int K, typename T>
__device__ __forceinline__ void gluon_level(const R4<T>* q, V4<T>* Gs, int gl) {
  constexpr int L = Lanes<NG>::L;
  constexpr int nblk = TTNG<NG>::FIRST[K + 1] - TTNG<NG>::FIRST[K];
  constexpr int items = nblk << K;
  constexpr int n3 = K - 1;
  constexpr int n4 = (K - 1) * (K - 2) / 2;
  for (int it = gl; it < items; it += L) {
    const int bl = it >> K;
    const unsigned c = unsigned(it) & ((1u << K) - 1u);
    const int b = TTNG<NG>::FIRST[K] + bl;
    const unsigned mb = blk_mask<NG>()[b];
    const unsigned H = pdep_mask<NG>(c, mb);
    V4<T> acc;
#pragma unroll
    for (int k = 0; k < 4; ++k) acc.c[k] = {T(0), T(0)};
    const uint8_t* t3 = o3_table<NG, K>() + bl * n3 * 2;
#pragma unroll
    for (int s = 0; s < n3; ++s) {
      const uint8_t rl = t3[2 * s], rr = t3[2 * s + 1];
      const V4<T> GL = load_block<NG, T>(Gs, rl, H), GR = load_block<NG, T>(Gs, rr, H);
      const R4<T> PL = block_momentum<NG, T>(q, blk_mask<NG>()[rl & 0x7f]);
      const R4<T> PR = block_momentum<NG, T>(q, blk_mask<NG>()[rr & 0x7f]);
      o3_sub(GL, GR, PL, PR, acc);
    }
    if constexpr (K >= 3) {
      const uint8_t* t4 = o4_table<NG, K>() + bl * n4 * 3;
#pragma unroll
      for (int s = 0; s < n4; ++s) {
        const V4<T> GL = load_block<NG, T>(Gs, t4[3 * s], H);
        const V4<T> GM = load_block<NG, T>(Gs, t4[3 * s + 1], H);
        const V4<T> GR = load_block<NG, T>(Gs, t4[3 * s + 2], H);
        o4_add(GL, GM, GR, acc);
      }
    }
    const R4<T> P = block_momentum<NG, T>(q, mb);
    const T inv = T(1) / mdot(P, P);
    V4<T> g;
#pragma unroll
    for (int k = 0; k < 4; ++k) g.c[k] = inv * acc.c[k];
    Gs[blk_off<NG>()[b] + c] = g;
  }
}

template <int NG, typename T>
__device__ __forceinline__ T lane_sum_dispatch(const R4<T>* q, const R4<T>& qtb, T m, T mw, const V4<T>* Gs,
                                               unsigned H, const S4<T>& vb, const S4<T>& ub0, const S4<T>& ub1) {
  cplx<T> J[TTNG<NG>::NPERM][2];
  if constexpr (NG == 2) return lane_colour_sum_2<T>(q, qtb, m, mw, Gs, H, vb, ub0, ub1, J);
  else if constexpr (NG == 3) return lane_colour_sum_3<T>(q, qtb, m, mw, Gs, H, vb, ub0, ub1, J);
  else return lane_colour_sum_4<T>(q, qtb, m, mw, Gs, H, vb, ub0, ub1, J);
}

// |M|^2 (without the normalisation MeParams::norm) of one event, computed by
// its lane group; p: physical momenta in MadGraph order.  Every lane of the
// warp must call this (the group synchronises with __syncwarp).
template <int NG, typename T>
__device__ __forceinline__ T group_me2(const T (&p)[NG + 2][4], V4<T>* Gs, int gl, T mt, T mw) {
  constexpr int L = Lanes<NG>::L;
  R4<T> q[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const int leg = g < 2 ? g : g + 2;
    const T s = g < 2 ? T(-1) : T(1);
#pragma unroll
    for (int c = 0; c < 4; ++c) q[g].v[c] = s * p[leg][c];
  }
  R4<T> qtb, pt;
#pragma unroll
  for (int c = 0; c < 4; ++c) { qtb.v[c] = p[3][c]; pt.v[c] = p[2][c]; }
  // level 1: polarisation vectors of every gluon, both helicities
  for (int it = gl; it < 2 * NG; it += L) {
    const int g = it >> 1;
    const int leg = g < 2 ? g : g + 2;
    R4<T> k;
#pragma unroll
    for (int c = 0; c < 4; ++c) k.v[c] = p[leg][c];
    Gs[2 * g + (it & 1)] = polarisation(k, (it & 1) ? 1 : -1, g >= 2);
  }
  __syncwarp();
  gluon_level<NG, 2, T>(q, Gs, gl);
  if constexpr (NG >= 3) { __syncwarp(); gluon_level<NG, 3, T>(q, Gs, gl); }
  if constexpr (NG >= 4) { __syncwarp(); gluon_level<NG, 4, T>(q, Gs, gl); }
  __syncwarp();
  const unsigned H = unsigned(gl) & ((1u << NG) - 1u);
  const int ltb = ((gl >> NG) & 1) ? 1 : -1;
  const S4<T> vb = v_out(qtb, mt, ltb);
  const S4<T> ub0 = ubar_out(pt, mt, -1);
  const S4<T> ub1 = ubar_out(pt, mt, 1);
  T part = lane_sum_dispatch<NG, T>(q, qtb, mt, mw, Gs, H, vb, ub0, ub1);
#pragma unroll
  for (int off = L / 2; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  __syncwarp();   // the group's shared store may be overwritten after this
  return part;
}

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;
constexpr int kTile = 128;

// ----------------------------------------------------------------------------
template <int NG, typename T>
__global__ void __launch_bounds__(kThreads) k_matrix_element(MeParams mp, int64_t n, const double* __restrict__ mom,
                                                             double* __restrict__ out) {
  constexpr int EPW = Lanes<NG>::EPW, L = Lanes<NG>::L, NEXT = Lanes<NG>::NEXT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V4<T>* Gs_all = reinterpret_cast<V4<T>*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int group = lane / L, gl = lane % L;
  V4<T>* Gs = Gs_all + (warp * EPW + group) * TTNG<NG>::NSTORE;
  const T mt = T(mp.mt), mw = T(mp.mw);
  for (int64_t base = (int64_t(blockIdx.x) * kWarps + warp) * EPW; base < n;
       base += int64_t(gridDim.x) * kWarps * EPW) {
    const int64_t ev = base + group;
    const bool ok = ev < n;
    const int64_t e = ok ? ev : base;
    T p[NEXT][4];
#pragma unroll
    for (int i = 0; i < NEXT; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) p[i][c] = T(mom[int64_t(i * 4 + c) * n + e]);
    const T v = group_me2<NG, T>(p, Gs, gl, mt, mw);
    if (ok && gl == 0) out[e] = double(v) * mp.norm;
  }
}

// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_sample(SampleParams sp, const double* __restrict__ edges_g, int64_t n,
                                                     uint64_t seed, int iter, double* __restrict__ mom,
                                                     double* __restrict__ wps, uint8_t* __restrict__ bins);

// Vegas accumulators of one CTA: [0] sum w, [1] sum w^2, [2 + j*nbins + b] sum w^2 in bin b of dim j
__device__ __forceinline__ void accumulate_event(double w, const uint8_t* b_ev, int ndim, int nbins, int stride,
                                                 double* sums, double* hist) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  double s1 = w, s2 = w * w;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_xor_sync(full, s1, off);
    s2 += __shfl_xor_sync(full, s2, off);
  }
  if (lane == 0) {
    atomicAdd(&sums[0], s1);
    atomicAdd(&sums[1], s2);
  }
  const double w2 = w * w;
  for (int j = 0; j < ndim; ++j) {
    const unsigned b = b_ev[j * stride];
    // lanes holding the same bin form a group; reduce it with a shuffle tree
    const unsigned peers = __match_any_sync(full, b);
    const unsigned below = peers & ((1u << lane) - 1u);
    const int rank = __popc(below);
    double v = w2;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
      // lane holding rank + s in the same group (or myself if none)
      unsigned m = peers & ~((lane == 31) ? 0xffffffffu : ((2u << lane) - 1u));
      for (int k = 1; k < s && m; ++k) m &= m - 1u;
      const int src = m ? (__ffs(m) - 1) : lane;
      const double o = __shfl_sync(full, v, src);
      if (m && (rank % (2 * s)) == 0) v += o;
    }
    if (rank == 0) atomicAdd(&hist[j * nbins + b], v);
  }
}

// Shared-memory layout of k_fused (bytes), shared by host and device.
template <int NG, typename T> struct FusedLayout {
  static constexpr int NEXT = NG + 2;
  static constexpr int EPW = Lanes<NG>::EPW;
  __host__ __device__ static size_t al(size_t x) { return (x + 15) & ~size_t(15); }
  __host__ __device__ static size_t edges(int, int) { return 0; }
  __host__ __device__ static size_t hist(int ndim, int nbins) { return al(edges(ndim, nbins) + sizeof(double) * ndim * (nbins + 1)); }
  __host__ __device__ static size_t sums(int ndim, int nbins) { return al(hist(ndim, nbins) + sizeof(double) * ndim * nbins); }
  __host__ __device__ static size_t pref(int ndim, int nbins) { return al(sums(ndim, nbins) + sizeof(double) * 2); }
  __host__ __device__ static size_t me2(int ndim, int nbins) { return al(pref(ndim, nbins) + sizeof(double) * kTile); }
  __host__ __device__ static size_t mom(int ndim, int nbins) { return al(me2(ndim, nbins) + sizeof(double) * kTile); }
  __host__ __device__ static size_t gs(int ndim, int nbins) { return al(mom(ndim, nbins) + sizeof(T) * kTile * NEXT * 4); }
  __host__ __device__ static size_t bins(int ndim, int nbins) {
    return al(gs(ndim, nbins) + sizeof(V4<T>) * kWarps * EPW * TTNG<NG>::NSTORE);
  }
  __host__ __device__ static size_t plist(int ndim, int nbins) { return al(bins(ndim, nbins) + size_t(ndim) * kTile); }
  __host__ __device__ static size_t total(int ndim, int nbins) { return al(plist(ndim, nbins) + sizeof(int) * (kTile + 4)); }
};

// Persistent fused kernel: each CTA walks tiles of kTile events.
//   phase 1 (thread per event): Philox -> Vegas -> luminosity -> RAMBO -> cuts
//   phase 2 (lane group per surviving event): |M|^2
//   phase 3 (thread per event): w = |M|^2 * prefactor, Vegas sums
// partials[blockIdx.x * nacc + k] receives the CTA's sums (nacc = 2 + ndim*nbins);
// counters[blockIdx.x * 2 + {0,1}] = events passing cuts, Newton misses.
template <int NG, typename T>
__global__ void __launch_bounds__(kThreads) k_fused(SampleParams sp, MeParams mp, const double* __restrict__ edges_g,
                                                    int64_t first_event, int64_t n, uint64_t seed, int iter,
                                                    double* __restrict__ partials,
                                                    unsigned long long* __restrict__ counters,
                                                    double* __restrict__ w_out) {
  using LY = FusedLayout<NG, T>;
  constexpr int EPW = Lanes<NG>::EPW, L = Lanes<NG>::L, NEXT = Lanes<NG>::NEXT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ndim = sp.ndim, nbins = sp.nbins;
  double* edges = reinterpret_cast<double*>(smem_raw + LY::edges(ndim, nbins));
  double* hist = reinterpret_cast<double*>(smem_raw + LY::hist(ndim, nbins));
  double* sums = reinterpret_cast<double*>(smem_raw + LY::sums(ndim, nbins));
  double* pref = reinterpret_cast<double*>(smem_raw + LY::pref(ndim, nbins));
  double* me2 = reinterpret_cast<double*>(smem_raw + LY::me2(ndim, nbins));
  T* mom = reinterpret_cast<T*>(smem_raw + LY::mom(ndim, nbins));
  V4<T>* Gs_all = reinterpret_cast<V4<T>*>(smem_raw + LY::gs(ndim, nbins));
  uint8_t* bins = smem_raw + LY::bins(ndim, nbins);
  int* plist = reinterpret_cast<int*>(smem_raw + LY::plist(ndim, nbins));
  int* pcount = plist + kTile;

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int group = lane / L, gl = lane % L;
  for (int i = t; i < ndim * (nbins + 1); i += kThreads) edges[i] = edges_g[i];
  for (int i = t; i < ndim * nbins; i += kThreads) hist[i] = 0.0;
  if (t < 2) sums[t] = 0.0;
  unsigned long long npass = 0, nfail = 0;
  V4<T>* Gs = Gs_all + (warp * EPW + group) * TTNG<NG>::NSTORE;
  const T mt = T(mp.mt), mw = T(mp.mw);
  __syncthreads();

  for (int64_t tile = blockIdx.x; tile * kTile < n; tile += gridDim.x) {
    if (t == 0) *pcount = 0;
    __syncthreads();
    const int64_t ev = tile * kTile + t;
    const bool valid = ev < n;
    int pass = 0;
    if (valid) {
      EventKin k;
      sample_event(sp, edges, seed, iter, uint64_t(first_event + ev), k);
#pragma unroll
      for (int i = 0; i < NEXT; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) mom[(t * NEXT + i) * 4 + c] = T(k.p[i][c]);
      pref[t] = k.prefactor;
      for (int j = 0; j < ndim; ++j) bins[j * kTile + t] = k.bins[j];
      pass = k.pass;
      npass += pass;
      nfail += k.newton_fail;
    } else {
      pref[t] = 0.0;
      for (int j = 0; j < ndim; ++j) bins[j * kTile + t] = 0;
    }
    me2[t] = 0.0;
    const unsigned bal = __ballot_sync(0xffffffffu, pass);
    int wbase = 0;
    if (lane == 0 && bal) wbase = atomicAdd(pcount, __popc(bal));
    wbase = __shfl_sync(0xffffffffu, wbase, 0);
    if (pass) plist[wbase + __popc(bal & ((1u << lane) - 1u))] = t;
    __syncthreads();

    const int np = *pcount;
    for (int base = warp * EPW; base < np; base += kWarps * EPW) {
      const int k = base + group;
      const bool ok = k < np;
      const int slot = plist[ok ? k : base];
      T p[NEXT][4];
#pragma unroll
      for (int i = 0; i < NEXT; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) p[i][c] = mom[(slot * NEXT + i) * 4 + c];
      const T v = group_me2<NG, T>(p, Gs, gl, mt, mw);
      if (ok && gl == 0) me2[slot] = double(v) * mp.norm;
    }
    __syncthreads();

    const double w = valid ? me2[t] * pref[t] : 0.0;
    if (w_out != nullptr && valid) w_out[ev] = w;
    accumulate_event(w, bins + t, ndim, nbins, kTile, sums, hist);
    __syncthreads();
  }
  const int nacc = 2 + ndim * nbins;
  double* dst = partials + int64_t(blockIdx.x) * nacc;
  for (int i = t; i < ndim * nbins; i += kThreads) dst[2 + i] = hist[i];
  if (t < 2) dst[t] = sums[t];
  // CTA totals of the counters
  for (int off = 16; off > 0; off >>= 1) {
    npass += __shfl_xor_sync(0xffffffffu, npass, off);
    nfail += __shfl_xor_sync(0xffffffffu, nfail, off);
  }
  __shared__ unsigned long long cnt[2];
  if (t < 2) cnt[t] = 0;
  __syncthreads();
  if (lane == 0) {
    atomicAdd(&cnt[0], npass);
    atomicAdd(&cnt[1], nfail);
  }
  __syncthreads();
  if (t < 2) counters[blockIdx.x * 2 + t] = cnt[t];
}

// host-side launch helpers (defined per gluon count)
template <int NG>
cudaError_t launch_matrix_element(int precision, const MeParams& mp, int64_t n, const double* mom, double* out,
                                  int grid, cudaStream_t s);
template <int NG>
cudaError_t launch_fused(int precision, const SampleParams& sp, const MeParams& mp, const double* edges,
                         int64_t first_event, int64_t n, uint64_t seed, int iter, double* partials,
                         unsigned long long* counters, double* w_out, int grid, cudaStream_t s);
template <int NG>
cudaError_t fused_config(int precision, int ndim, int nbins, size_t* smem, int* ctas_per_sm);
template <int NG>
cudaError_t me_config(int precision, size_t* smem, int* ctas_per_sm);

cudaError_t launch_sample(const SampleParams& sp, const double* edges, int64_t n, uint64_t seed, int iter,
                          double* mom, double* wps, uint8_t* bins, cudaStream_t s);
// totals: [0] sum w, [1] sum w^2, [2 + j*nbins + b] histogram, [nacc] passing events, [nacc+1] Newton misses
cudaError_t launch_reduce(const double* partials, const unsigned long long* counters, int nblocks, int ndim, int nbins,
                          double* totals, cudaStream_t s);
// result: [0] sum w, [1] sum w^2, [2] I_k, [3] sigma_k^2, [4] passing events, [5] Newton misses
cudaError_t launch_finish(const double* totals, int ndim, int nbins, int64_t n_total, int refine, double* edges,
                          double* result, cudaStream_t s);
cudaError_t launch_fma_peak(int precision, int blocks, int iters, float* sink, cudaStream_t s);

}  // namespace mf

#define MF_INSTANTIATE(NG)                                                                                        \
  namespace mf {                                                                                                  \
  template <>                                                                                                     \
  cudaError_t me_config<NG>(int precision, size_t* smem, int* ctas) {                                             \
    cudaError_t e;                                                                                                \
    if (precision == 0) {                                                                                         \
      *smem = sizeof(V4<double>) * kWarps * Lanes<NG>::EPW * TTNG<NG>::NSTORE;                                    \
      e = cudaFuncSetAttribute(k_matrix_element<NG, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem)); \
      if (e != cudaSuccess) return e;                                                                             \
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_matrix_element<NG, double>, kThreads, *smem);  \
    }                                                                                                             \
    *smem = sizeof(V4<float>) * kWarps * Lanes<NG>::EPW * TTNG<NG>::NSTORE;                                       \
    e = cudaFuncSetAttribute(k_matrix_element<NG, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem)); \
    if (e != cudaSuccess) return e;                                                                               \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_matrix_element<NG, float>, kThreads, *smem);     \
  }                                                                                                               \
  template <>                                                                                                     \
  cudaError_t launch_matrix_element<NG>(int precision, const MeParams& mp, int64_t n, const double* mom,          \
                                        double* out, int grid, cudaStream_t s) {                                  \
    if (precision == 0) {                                                                                         \
      const size_t sm = sizeof(V4<double>) * kWarps * Lanes<NG>::EPW * TTNG<NG>::NSTORE;                          \
      k_matrix_element<NG, double><<<grid, kThreads, sm, s>>>(mp, n, mom, out);                                   \
    } else {                                                                                                      \
      const size_t sm = sizeof(V4<float>) * kWarps * Lanes<NG>::EPW * TTNG<NG>::NSTORE;                           \
      k_matrix_element<NG, float><<<grid, kThreads, sm, s>>>(mp, n, mom, out);                                    \
    }                                                                                                             \
    return cudaGetLastError();                                                                                    \
  }                                                                                                               \
  template <>                                                                                                     \
  cudaError_t fused_config<NG>(int precision, int ndim, int nbins, size_t* smem, int* ctas) {                     \
    cudaError_t e;                                                                                                \
    if (precision == 0) {                                                                                         \
      *smem = FusedLayout<NG, double>::total(ndim, nbins);                                                        \
      e = cudaFuncSetAttribute(k_fused<NG, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem));     \
      if (e != cudaSuccess) return e;                                                                             \
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_fused<NG, double>, kThreads, *smem);           \
    }                                                                                                             \
    *smem = FusedLayout<NG, float>::total(ndim, nbins);                                                           \
    e = cudaFuncSetAttribute(k_fused<NG, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem));        \
    if (e != cudaSuccess) return e;                                                                               \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_fused<NG, float>, kThreads, *smem);              \
  }                                                                                                               \
  template <>                                                                                                     \
  cudaError_t launch_fused<NG>(int precision, const SampleParams& sp, const MeParams& mp, const double* edges,    \
                               int64_t first_event, int64_t n, uint64_t seed, int iter, double* partials,         \
                               unsigned long long* counters, double* w_out, int grid, cudaStream_t s) {           \
    if (precision == 0) {                                                                                         \
      const size_t sm = FusedLayout<NG, double>::total(sp.ndim, sp.nbins);                                        \
      k_fused<NG, double><<<grid, kThreads, sm, s>>>(sp, mp, edges, first_event, n, seed, iter, partials,       \
                                                     counters, w_out);                                          \
    } else {                                                                                                      \
      const size_t sm = FusedLayout<NG, float>::total(sp.ndim, sp.nbins);                                         \
      k_fused<NG, float><<<grid, kThreads, sm, s>>>(sp, mp, edges, first_event, n, seed, iter, partials,        \
                                                    counters, w_out);                                           \
    }                                                                                                             \
    return cudaGetLastError();                                                                                    \
  }                                                                                                               \
  }
