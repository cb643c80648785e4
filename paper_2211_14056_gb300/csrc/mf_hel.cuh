// Helicity sampling for a top pair plus NG gluons: |M|^2 of ONE helicity
// configuration per event (the gluons' and the antitop's helicities, both top
// helicities summed), the estimator of the helicity sum being 2^(NG+1) times
// that value for a configuration drawn uniformly.  arXiv:2211.14056 (Sec. 2)
// sums the helicities inside its matrix-element operator; drawing one per
// event is the MadEvent/MadFlow alternative that trades variance for work.
//
// Work split: a group of four lanes per event (eight events per warp).  The
// event's colour-ordered gluon sub-currents G(B) exist for one helicity
// pattern only, so each block B holds a single current (34 for NG = 4, about
// 1 KB in FP32), built level by level by the group; lane c < NG then walks the
// quark-line subtree whose last gluon is c (the level-1 suffix (c)), which
// gives the colour orderings ending in c; the four lanes share the colour
// forms J^dagger (D C) J of the two top helicities, each lane half of one
// form (a gluon relabelling that leaves D C invariant maps one half onto the
// other: colour_form_orbit in mf_gen_ttng.cuh).  The summed kernels' tables
// (mf_gen_ttng.cuh) serve unchanged: a block reference's stored offset is
// mapped to the block's index (hel_blk).
#pragma once
#include "mf_kernels.cuh"

namespace mf {

constexpr int kHelGroup = 4;                   // lanes per event
constexpr int kHelEPW = 32 / kHelGroup;        // events per warp

// Shared memory of one event: G[NBLK] (block-major, one V4 per block), the
// mask table, the amplitudes J[sigma][top helicity].  16 bytes of padding
// shift consecutive events across the banks.
template <int NG, typename T> struct HelMem {
  static constexpr int NBLK = TTNG<NG>::NBLK, NP = TTNG<NG>::NPERM;
  static constexpr size_t al(size_t x) { return (x + 15) & ~size_t(15); }
  static constexpr size_t mt_off = al(sizeof(V4<T>) * NBLK);
  static constexpr size_t j_off = al(mt_off + MaskTab<NG, T>::bytes);
  static constexpr size_t event_bytes = al(j_off + sizeof(cplx<T>) * NP * 2) + 16;
  static constexpr size_t warp_bytes = event_bytes * kHelEPW;
};

// Offset of the first stored current of the blocks of length len in the
// summed layout (each block of length k stores 2^k currents), packed 16 bits
// per length from length 1 up; and the index of the first block of each
// length, 8 bits each.
template <int NG> constexpr uint64_t hel_off0_packed() {
  uint64_t r = 0;
  int o = 0;
  for (int len = 1; len <= NG; ++len) {
    r |= uint64_t(o) << (16 * (len - 1));
    o += (TTNG<NG>::FIRST[len + 1] - TTNG<NG>::FIRST[len]) << len;
  }
  return r;
}
template <int NG> constexpr uint64_t hel_first_packed() {
  uint64_t r = 0;
  for (int len = 1; len <= NG; ++len) r |= uint64_t(TTNG<NG>::FIRST[len]) << (8 * (len - 1));
  return r;
}

// Index of a referenced block: its length is the popcount of its gluon mask,
// and within a length the stored offsets advance by 2^len per block.
template <int NG> __device__ __forceinline__ int hel_blk(uint16_t ref) {
  constexpr uint64_t off0 = hel_off0_packed<NG>(), first = hel_first_packed<NG>();
  const int len = __popc(ref_mask(ref));
  const int o0 = int((off0 >> (16 * (len - 1))) & 0xffffu);
  const int f = int((first >> (8 * (len - 1))) & 0xffu);
  return f + ((ref_off(ref) - o0) >> len);
}

template <int NG, typename T> __device__ __forceinline__ V4<T> hel_load(const V4<T>* G, uint16_t ref) {
  return G[hel_blk<NG>(ref)];
}

// one level (block length K) of the sub-currents for the event's helicities
template <int NG, int K, typename T>
__device__ __forceinline__ void hel_gluon_level(const MaskTab<NG, T>& mt, V4<T>* G, int gl) {
  constexpr int nblk = TTNG<NG>::FIRST[K + 1] - TTNG<NG>::FIRST[K];
  constexpr int n3 = K - 1;
  constexpr int n4 = (K - 1) * (K - 2) / 2;
#pragma unroll 1
  for (int bl = gl; bl < nblk; bl += kHelGroup) {
    const int b = TTNG<NG>::FIRST[K] + bl;
    const unsigned mb = blk_mask<NG>()[b];
    V4<T> acc;
#pragma unroll
    for (int k = 0; k < 4; ++k) acc.c[k] = {T(0), T(0)};
    const uint16_t* t3 = o3_table<NG, K>() + bl * n3 * 2;
#pragma unroll
    for (int s = 0; s < n3; ++s) {
      const uint16_t rl = t3[2 * s], rr = t3[2 * s + 1];
      const V4<T> GL = hel_load<NG, T>(G, rl), GR = hel_load<NG, T>(G, rr);
      o3_sub(GL, GR, mt.qsum[ref_mask(rl)], mt.qsum[ref_mask(rr)], (ref_neg(rl) != ref_neg(rr)) ? T(-1) : T(1), acc);
    }
    if constexpr (K >= 3) {
      const uint16_t* t4 = o4_table<NG, K>() + bl * n4 * 3;
#pragma unroll
      for (int s = 0; s < n4; ++s) {
        const uint16_t r0 = t4[3 * s], r1 = t4[3 * s + 1], r2 = t4[3 * s + 2];
        o4_add(hel_load<NG, T>(G, r0), hel_load<NG, T>(G, r1), hel_load<NG, T>(G, r2),
               (ref_neg(r0) ^ ref_neg(r1) ^ ref_neg(r2)) ? T(-1) : T(1), acc);
      }
    }
    const T inv = mt.ginv[mb];
    V4<T> g;
#pragma unroll
    for (int k = 0; k < 4; ++k) g.c[k] = inv * acc.c[k];
    G[b] = g;
  }
}

// Per-lane context of the quark-line subtree walk.
template <typename T> struct HelCtx {
  const V4<T>* G;       // this event's sub-currents
  const R4<T>* Ptab;    // -(q_tbar + sum of the gluon momenta in mask), by mask
  const cplx<T>* qf;    // heavy-quark propagator factor, by mask
  S4<T> ub0, ub1;       // ubar(t) for top helicity -1, +1
  T m;
  cplx<T>* J;           // this event's amplitudes [sigma * 2 + top helicity]
};

template <int NG, typename T> __device__ __forceinline__ V4<T> hel_block(const HelCtx<T>& cx, uint16_t ref) {
  V4<T> g = hel_load<NG, T>(cx.G, ref);
  if (ref_neg(ref)) g = neg(g);
  return g;
}

// The suffix `path` of level LV (|S| = LV) and everything below it:
// R(S) = -(P_S-slash + m)/(P_S^2 - m^2 + i m Gamma) sum_m G(S[:m])-slash R(S[m:]),
// and at level NG - 1 the amplitude J_sigma = ubar(t) sum_m G(sigma[:m])-slash
// R(sigma[m:]) of the one completion sigma = (a,) + S, for both top helicities.
template <int NG, int LV, typename T>
__device__ __forceinline__ void hel_path(int path, S4<T> (&R)[NG], const HelCtx<T>& cx) {
  using PT = Paths<NG>;
  const uint8_t msk = PT::template mask<LV>(path);
  S4<T> X = apply(make_slash(hel_block<NG, T>(cx, PT::template blk<LV>(path, 0))), R[LV - 1]);
#pragma unroll
  for (int m = 1; m < LV; ++m)
    apply_acc(make_slash(hel_block<NG, T>(cx, PT::template blk<LV>(path, m))), R[LV - 1 - m], X);
  R[LV] = quark_prop_f(cx.Ptab[msk], cx.m, cx.qf[msk], X);
  if constexpr (LV < NG - 1) {
    const int first = PT::template first<LV + 1>(path);
#pragma unroll 1
    for (int k = 0; k < NG - LV; ++k) hel_path<NG, LV + 1, T>(first + k, R, cx);
  } else {
    S4<T> W = apply(make_slash(hel_block<NG, T>(cx, PT::final_blk(path, 0))), R[NG - 1]);
#pragma unroll
    for (int m = 1; m < NG; ++m)
      apply_acc(make_slash(hel_block<NG, T>(cx, PT::final_blk(path, m))), R[NG - 1 - m], W);
    const int sig = PT::final_sigma(path);
    cx.J[sig * 2 + 0] = rowdot(cx.ub0, W);
    cx.J[sig * 2 + 1] = rowdot(cx.ub1, W);
  }
}

// |M_h|^2 summed over the top's helicities (without MeParams::norm) of one
// event for the configuration `hel` (bit g < NG: gluon g has helicity +1, the
// gluons in MadGraph order; bit NG: antitop helicity +1), computed by the
// event's four lanes (gl = 0..3) in the event's shared memory `em` (HelMem
// layout).  Every lane of the warp must call this (__syncwarp inside); all four
// lanes of the group return the value.
template <int NG, typename T>
__device__ __forceinline__ T hel_me2(const T (&p)[NG + 2][4], unsigned hel, unsigned char* em, int gl, T mt, T mw) {
  using HM = HelMem<NG, T>;
  constexpr int NP = TTNG<NG>::NPERM;
  V4<T>* G = reinterpret_cast<V4<T>*>(em);
  const MaskTab<NG, T> mtab(em + HM::mt_off);
  cplx<T>* J = reinterpret_cast<cplx<T>*>(em + HM::j_off);
  R4<T> q[NG];
  gluon_momenta<NG, T>(p, q);
  R4<T> qtb, pt;
#pragma unroll
  for (int c = 0; c < 4; ++c) { qtb.v[c] = p[3][c]; pt.v[c] = p[2][c]; }
#pragma unroll 1
  for (int msk = gl; msk < (1 << NG); msk += kHelGroup) mask_entry<NG, T>(q, qtb, msk, mtab, mt, mw);
  // level 1: the polarisation vector of each gluon's drawn helicity (gluon g
  // by lane g mod 4; the loop is unrolled so that p is indexed by constants)
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    if ((g & (kHelGroup - 1)) == gl) {
      const int leg = g < 2 ? g : g + 2;
      R4<T> k;
#pragma unroll
      for (int c = 0; c < 4; ++c) k.v[c] = p[leg][c];
      G[g] = polarisation(k, ((hel >> g) & 1u) ? 1 : -1, g >= 2);
    }
  }
  __syncwarp();
  hel_gluon_level<NG, 2, T>(mtab, G, gl);
  if constexpr (NG >= 3) { __syncwarp(); hel_gluon_level<NG, 3, T>(mtab, G, gl); }
  if constexpr (NG >= 4) { __syncwarp(); hel_gluon_level<NG, 4, T>(mtab, G, gl); }
  __syncwarp();
  if (gl < NG) {
    HelCtx<T> cx;
    cx.G = G;
    cx.Ptab = mtab.ptab;
    cx.qf = mtab.qf;
    cx.ub0 = ubar_out(pt, mt, -1);
    cx.ub1 = ubar_out(pt, mt, 1);
    cx.m = mt;
    cx.J = J;
    S4<T> R[NG];
    R[0] = v_out(qtb, mt, ((hel >> NG) & 1u) ? 1 : -1);
    hel_path<NG, 1, T>(gl, R, cx);
  }
  __syncwarp();   // every ordering's amplitudes are in shared memory
  // colour forms: lane gl takes top helicity gl & 1 and, for gl >> 1 = 1, the
  // orderings relabelled by the gluon symmetry that leaves D C invariant;
  // the same half of the quadratic form (colour_form_orbit) on the two data
  // sets adds up to the helicity's form, so the four lanes share the work
  const int th = gl & 1, rel = gl >> 1;
  cplx<T> Jl[NP];
#pragma unroll
  for (int sg = 0; sg < NP; ++sg) Jl[sg] = J[(rel ? ColourPerm<NG>::at(sg) : sg) * 2 + th];
  T part = T(2) * colour_form_orbit<T>(Jl);
  part += __shfl_xor_sync(0xffffffffu, part, 1);
  part += __shfl_xor_sync(0xffffffffu, part, 2);
  __syncwarp();   // the event's shared memory may be overwritten after this
  return part;
}

// The helicity stream's word of global event ev: word 0 of the third Philox
// stream (key as the Vegas uniforms', counter (ev & 0xffffffff, ev >> 32, 1, 1)).
__device__ __forceinline__ uint32_t helicity_word(uint64_t seed, int iter, uint64_t ev) {
  const uint2 key = make_uint2(uint32_t(seed), uint32_t(seed >> 32) ^ uint32_t(iter));
  return philox4x32_10(make_uint4(uint32_t(ev), uint32_t(ev >> 32), 1u, 1u), key).x;
}

// The configuration drawn by word w0 from the thresholds T[0..H] (T[0] = 0,
// T[H] = 2^32, non-decreasing): h = max{h : T[h] <= w0}, by bisection.  With
// uniform thresholds this is the top NG + 1 bits of w0.
template <int NG> __device__ __forceinline__ unsigned helicity_draw(uint32_t w0, const unsigned long long* T) {
  constexpr int H = 2 << NG;
  unsigned lo = 0;
#pragma unroll
  for (int step = H / 2; step > 0; step >>= 1)
    if (T[lo + step] <= (unsigned long long)w0) lo += step;
  return lo;
}

// ----------------------------------------------------------------------------
// |M_h|^2 of given momenta (SoA [NG + 2][4][n]) and configurations hel[n]
// (only the low NG + 1 bits are read); out[e] = |M_h|^2 * MeParams::norm.
template <int NG, typename T>
__global__ void __launch_bounds__(kThreads) k_matrix_element_hel(MeParams mp, int64_t n, const double* __restrict__ mom,
                                                                 const int* __restrict__ hel, double* __restrict__ out) {
  constexpr int NEXT = NG + 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int group = lane / kHelGroup, gl = lane % kHelGroup;
  unsigned char* em = smem_raw + size_t(warp * kHelEPW + group) * HelMem<NG, T>::event_bytes;
  const T mt = T(mp.mt), mw = T(mp.mw);
  for (int64_t base = (int64_t(blockIdx.x) * kWarps + warp) * kHelEPW; base < n;
       base += int64_t(gridDim.x) * kWarps * kHelEPW) {
    const int64_t ev = base + group;
    const bool ok = ev < n;
    const int64_t e = ok ? ev : base;
    T p[NEXT][4];
#pragma unroll
    for (int i = 0; i < NEXT; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) p[i][c] = T(mom[int64_t(i * 4 + c) * n + e]);
    const unsigned h = unsigned(hel[e]) & ((2u << NG) - 1u);
    const T v = hel_me2<NG, T>(p, h, em, gl, mt, mw);
    if (ok && gl == 0) out[e] = double(v) * mp.norm;
  }
}

// Shared memory of k_me_acc_hel: the CTA's Vegas histogram and sums, the
// draw's thresholds and the per-configuration sums of squared weights, then
// the warps' events.
constexpr int kHelMaxConfigs = 32;
template <int NG, typename T> struct HelAccLayout {
  __host__ __device__ static size_t al(size_t x) { return (x + 15) & ~size_t(15); }
  __host__ __device__ static size_t sums(int nacc) { return al(sizeof(double) * (nacc - 2)); }
  __host__ __device__ static size_t thr(int nacc) { return al(sums(nacc) + sizeof(double) * 2); }
  __host__ __device__ static size_t hsq(int nacc) { return al(thr(nacc) + sizeof(unsigned long long) * (kHelMaxConfigs + 1)); }
  __host__ __device__ static size_t warps(int nacc) { return al(hsq(nacc) + sizeof(double) * kHelMaxConfigs); }
  __host__ __device__ static size_t total(int nacc) { return warps(nacc) + HelMem<NG, T>::warp_bytes * kWarps; }
};

// |M|^2 estimates of the listed events of one record chunk with one sampled
// helicity configuration each, weights w = |M_h|^2 norm * prefactor / p_h,
// p_h = (T[h+1] - T[h]) / 2^32 (2^(NG+1) |M_h|^2 ... with uniform
// thresholds), and the Vegas sums (as k_me_acc).  The configuration of the
// chunk's event e is drawn for global event first_event + e from the
// thresholds hel_T[0..2^(NG+1)].  With hel_sq given, hel_sq[blockIdx.x * 32 + h]
// receives (accumulate = 0) or adds (1) the CTA's sum of w^2 over the events
// drawn in configuration h (the refinement's input).
template <int NG, typename T>
__global__ void __launch_bounds__(kThreads, 3)
    k_me_acc_hel(MeParams mp, int ndim, int nbins, RecordView<T> rec, int accumulate, double* __restrict__ partials,
                 unsigned long long* __restrict__ counters, double* __restrict__ w_out, uint64_t seed, int iter,
                 int64_t first_event, const unsigned long long* __restrict__ hel_T, double* __restrict__ hel_sq) {
  constexpr int H = 2 << NG;
  using LY = HelAccLayout<NG, T>;
  constexpr int NEXT = NG + 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nacc = 2 + ndim * nbins;
  double* hist = reinterpret_cast<double*>(smem_raw);
  double* sums = reinterpret_cast<double*>(smem_raw + LY::sums(nacc));
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int group = lane / kHelGroup, gl = lane % kHelGroup;
  unsigned long long* thr = reinterpret_cast<unsigned long long*>(smem_raw + LY::thr(nacc));
  double* hsq = reinterpret_cast<double*>(smem_raw + LY::hsq(nacc));
  unsigned char* em = smem_raw + LY::warps(nacc) + size_t(warp * kHelEPW + group) * HelMem<NG, T>::event_bytes;
  for (int i = t; i < ndim * nbins; i += kThreads) hist[i] = 0.0;
  if (t < 2) sums[t] = 0.0;
  if (t <= H) thr[t] = hel_T[t];
  if (t < H) hsq[t] = 0.0;
  const T mt = T(mp.mt), mw = T(mp.mw);
  const unsigned full = 0xffffffffu;
  const int64_t npass = rec.count[0];
  double s1 = 0.0, s2 = 0.0;
  __syncthreads();

  const int64_t stride = int64_t(gridDim.x) * kWarps * kHelEPW;
  for (int64_t base = (int64_t(blockIdx.x) * kWarps + warp) * kHelEPW; base < npass; base += stride) {
    const int64_t k = base + group;
    const bool ok = k < npass;
    const int64_t e = rec.list[ok ? k : base];
    T p[NEXT][4];
    const T rs = rec.rs[e];
    p[0][0] = T(0.5) * rs; p[0][1] = T(0); p[0][2] = T(0); p[0][3] = T(0.5) * rs;
    p[1][0] = T(0.5) * rs; p[1][1] = T(0); p[1][2] = T(0); p[1][3] = T(-0.5) * rs;
#pragma unroll
    for (int i = 0; i < NG; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) p[2 + i][c] = rec.mom[int64_t(i * 4 + c) * rec.C + e];
    const unsigned h = helicity_draw<NG>(helicity_word(seed, iter, uint64_t(first_event + e)), thr);
    const T v = hel_me2<NG, T>(p, h, em, gl, mt, mw);
    if (ok) {
      // 1 / p_h = 2^32 / (T[h+1] - T[h]), exact for the uniform thresholds
      const double w = double(v) * mp.norm * rec.pref[e] * (4294967296.0 / double(thr[h + 1] - thr[h]));
      if (gl == 0) {
        s1 += w;
        s2 += w * w;
        if (w_out != nullptr) w_out[e] = w;
        if (hel_sq != nullptr) atomicAdd(&hsq[h], w * w);
      }
      for (int j = gl; j < ndim; j += kHelGroup)
        atomicAdd(&hist[j * nbins + rec.flag[int64_t(j) * rec.C + e]], w * w);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_xor_sync(full, s1, off);
    s2 += __shfl_xor_sync(full, s2, off);
  }
  if (lane == 0) {
    atomicAdd(&sums[0], s1);
    atomicAdd(&sums[1], s2);
  }
  __syncthreads();
  double* dst = partials + int64_t(blockIdx.x) * nacc;
  for (int i = t; i < ndim * nbins; i += kThreads) dst[2 + i] = (accumulate ? dst[2 + i] : 0.0) + hist[i];
  if (t < 2) dst[t] = (accumulate ? dst[t] : 0.0) + sums[t];
  if (t < 2) {
    const unsigned long long c = blockIdx.x == 0 ? (unsigned long long)rec.count[t] : 0ull;
    counters[blockIdx.x * 2 + t] = (accumulate ? counters[blockIdx.x * 2 + t] : 0ull) + c;
  }
  if (hel_sq != nullptr && t < H) {
    double* d = hel_sq + int64_t(blockIdx.x) * kHelMaxConfigs + t;
    *d = (accumulate ? *d : 0.0) + hsq[t];
  }
}

// host-side helpers (mf_hel.cu), NG = 2, 3, 4; precision 0: FP64, 1: FP32
cudaError_t hel_me_config(int ng, int precision, size_t* smem, int* ctas_per_sm);
cudaError_t launch_matrix_element_hel(int ng, int precision, const MeParams& mp, int64_t n, const double* mom,
                                      const int* hel, double* out, int grid, cudaStream_t s);
cudaError_t hel_acc_config(int ng, int precision, int ndim, int nbins, size_t* smem, int* ctas_per_sm);
// one record chunk: k_sample_rec, then k_me_acc_hel (ev: 3 events as launch_chunk);
// hel_T: the draw's thresholds (device), hel_sq: per-CTA sums of squared
// weights by configuration, [grid][32] (device, may be null)
cudaError_t launch_chunk_hel(int ng, int precision, const SampleParams& sp, const MeParams& mp, const double* edges,
                             int64_t first_event, int64_t n, int64_t C, void* rec_base, uint64_t seed, int iter,
                             int accumulate, double* partials, unsigned long long* counters, double* w_out, int grid,
                             cudaStream_t s, cudaEvent_t* ev, const unsigned long long* hel_T, double* hel_sq);
// the configurations' sums of squared weights over the CTAs (fixed order) into
// S[0..H-1], then (refine) the refined thresholds T[0..H]
cudaError_t launch_hel_reduce(const double* hel_sq, int nblocks, int n_configs, double* S, cudaStream_t s);
cudaError_t launch_hel_refine(const double* S, int n_configs, unsigned long long* T, cudaStream_t s);
// thresholds of probabilities p[0..H-1] (host): T_h = floor(2^32 (p_0 + ... + p_{h-1})),
// the partial sums added in order; T_0 = 0, T_H = 2^32
void hel_thresholds(const double* p, int n_configs, unsigned long long* T);
constexpr double kHelRefineFloor = 0.1;   // the share of the uniform probabilities kept by a refinement

}  // namespace mf
