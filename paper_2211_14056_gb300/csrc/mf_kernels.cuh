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
#include <type_traits>

#include "mf_device.cuh"
#include "mf_f32x2.cuh"
#include "mf_gen_ttng.cuh"
#include "mf_sample.cuh"

namespace mf {

struct MeParams {
  double mt, mw;     // top mass, mass * width
  double norm;       // g^(2 NG) / (spin-colour average * identical-particle factor * colour denominator)
  int colour_tc;     // 1: FP32 colour sum on the tensor cores (MF_FP32_TC)
  int chan;          // two-quark-line processes: which subprocess (beams, crossing) the amplitude serves
};

// MeParams::chan of the two-quark-line amplitude (mf_kernels_uux.cu): u u~, u~ u,
// u g, g u, u~ g, g u~ initial states
constexpr int kChanQQB = 0, kChanQBQ = 1, kChanQG = 2, kChanGQ = 3, kChanQBG = 4, kChanGQB = 5;

// The FP32 four-gluon quark line walks both antitop helicities of a lane as
// packed pairs (quark_walk_paired4_x2); false restores the scalar walk.
constexpr bool kPackedWalk = true;

template <int NG> struct Lanes {
  static constexpr int L = 2 << NG;        // lanes per event
  static constexpr int EPW = 32 / L;       // events per warp
  static constexpr int NEXT = NG + 2;
};

// Bit deposit / extract on the gluon-helicity masks (at most 4 gluons) by
// table: nibble x of kPdep4[m] is x's bits deposited at the set bits of m
// (ascending), nibble x of kPext4[m] is the bits of x at the set bits of m,
// packed.  One constant load, a shift and a mask replace a loop over the bits.
constexpr uint64_t nibble_table(unsigned m, bool deposit) {
  uint64_t t = 0;
  for (unsigned x = 0; x < 16; ++x) {
    unsigned r = 0, j = 0;
    for (unsigned g = 0; g < 4; ++g)
      if ((m >> g) & 1u) {
        if (deposit) r |= ((x >> j) & 1u) << g;
        else r |= ((x >> g) & 1u) << j;
        ++j;
      }
    t |= uint64_t(r) << (4 * x);
  }
  return t;
}
static __constant__ uint64_t kPdep4[16] = {
    nibble_table(0, true),  nibble_table(1, true),  nibble_table(2, true),  nibble_table(3, true),
    nibble_table(4, true),  nibble_table(5, true),  nibble_table(6, true),  nibble_table(7, true),
    nibble_table(8, true),  nibble_table(9, true),  nibble_table(10, true), nibble_table(11, true),
    nibble_table(12, true), nibble_table(13, true), nibble_table(14, true), nibble_table(15, true)};
static __constant__ uint64_t kPext4[16] = {
    nibble_table(0, false),  nibble_table(1, false),  nibble_table(2, false),  nibble_table(3, false),
    nibble_table(4, false),  nibble_table(5, false),  nibble_table(6, false),  nibble_table(7, false),
    nibble_table(8, false),  nibble_table(9, false),  nibble_table(10, false), nibble_table(11, false),
    nibble_table(12, false), nibble_table(13, false), nibble_table(14, false), nibble_table(15, false)};

template <int NG>
__device__ __forceinline__ unsigned pdep_mask(unsigned c, unsigned mask) {
  static_assert(NG <= 4, "helicity tables cover at most 4 gluons");
  return unsigned(kPdep4[mask] >> (4 * c)) & 15u;
}

template <int NG>
__device__ __forceinline__ unsigned pext_mask(unsigned H, unsigned mask) {
  static_assert(NG <= 4, "helicity tables cover at most 4 gluons");
  return unsigned(kPext4[mask] >> (4 * H)) & 15u;
}

// Per-event quantities that depend on a subset (mask) of the gluons but on no
// helicity, computed once per event by the lane group and kept in shared
// memory: ptab = -(q_tbar + K), qsum = K = sum of the gluon momenta in the
// mask (incoming ones negated), ginv = 1/K^2 (masks of two or more gluons),
// qf = -1/(P^2 - m^2 + i m Gamma) for P = q_tbar + K, the heavy-quark
// propagator factor of the suffix with these gluons.
template <int NG, typename T> struct MaskTab {
  static constexpr int M = 1 << NG;
  static constexpr size_t bytes = size_t(M) * (2 * sizeof(R4<T>) + sizeof(T) + sizeof(cplx<T>));
  R4<T>* ptab;
  R4<T>* qsum;
  T* ginv;
  cplx<T>* qf;
  __device__ __forceinline__ explicit MaskTab(unsigned char* base)
      : ptab(reinterpret_cast<R4<T>*>(base)),
        qsum(reinterpret_cast<R4<T>*>(base + M * sizeof(R4<T>))),
        ginv(reinterpret_cast<T*>(base + 2 * M * sizeof(R4<T>))),
        qf(reinterpret_cast<cplx<T>*>(base + 2 * M * sizeof(R4<T>) + M * sizeof(T))) {}
};

// The sub-currents of one event are stored component-major, Gs[mu * NSTORE + pos]:
// the lanes of a warp read 2^k consecutive positions of one block at a time,
// which then fall into distinct banks.
template <int NG, typename T>
__device__ __forceinline__ V4<T> gs_load(const cplx<T>* Gs, int pos) {
  V4<T> g;
#pragma unroll
  for (int k = 0; k < 4; ++k) g.c[k] = Gs[k * TTNG<NG>::NSTORE + pos];
  return g;
}

template <int NG, typename T>
__device__ __forceinline__ void gs_store(cplx<T>* Gs, int pos, const V4<T>& g) {
#pragma unroll
  for (int k = 0; k < 4; ++k) Gs[k * TTNG<NG>::NSTORE + pos] = g.c[k];
}

// Block references (generated tables): shared-memory offset of the block's
// stored currents in bits 0-8, gluon mask in bits 9-12, reversal sign in bit 13.
__device__ __forceinline__ int ref_off(uint16_t ref) { return ref & 511; }
__device__ __forceinline__ unsigned ref_mask(uint16_t ref) { return (ref >> 9) & 15u; }
__device__ __forceinline__ bool ref_neg(uint16_t ref) { return (ref >> 13) & 1u; }

// stored currents of a block for helicities H, without the reversal sign
template <int NG, typename T>
__device__ __forceinline__ V4<T> load_block(const cplx<T>* Gs, uint16_t ref, unsigned H) {
  return gs_load<NG, T>(Gs, ref_off(ref) + pext_mask<NG>(H, ref_mask(ref)));
}

// one level (block length K) of the colour-ordered gluon currents
template <int NG, int K, typename T>
__device__ __forceinline__ void gluon_level(const MaskTab<NG, T>& mt, cplx<T>* Gs, int gl) {
  constexpr int L = Lanes<NG>::L;
  constexpr int nblk = TTNG<NG>::FIRST[K + 1] - TTNG<NG>::FIRST[K];
  constexpr int items = nblk << K;
  constexpr int n3 = K - 1;
  constexpr int n4 = (K - 1) * (K - 2) / 2;
  // one item per loop body: two inlined copies (unroll 2) ran 5% slower over
  // the whole FP32 iteration (the kernel's hot code outgrows the
  // instruction cache)
#pragma unroll 1
  for (int it = gl; it < items; it += L) {
    const int bl = it >> K;
    const unsigned c = unsigned(it) & ((1u << K) - 1u);
    const int b = TTNG<NG>::FIRST[K] + bl;
    const unsigned mb = blk_mask<NG>()[b];
    const unsigned H = pdep_mask<NG>(c, mb);
    V4<T> acc;
#pragma unroll
    for (int k = 0; k < 4; ++k) acc.c[k] = {T(0), T(0)};
    const uint16_t* t3 = o3_table<NG, K>() + bl * n3 * 2;
#pragma unroll
    for (int s = 0; s < n3; ++s) {
      const uint16_t rl = t3[2 * s], rr = t3[2 * s + 1];
      const V4<T> GL = load_block<NG, T>(Gs, rl, H), GR = load_block<NG, T>(Gs, rr, H);
      const R4<T> PL = mt.qsum[ref_mask(rl)];
      const R4<T> PR = mt.qsum[ref_mask(rr)];
      // the vertex is bilinear: the blocks' reversal signs multiply it
      o3_sub(GL, GR, PL, PR, (ref_neg(rl) != ref_neg(rr)) ? T(-1) : T(1), acc);
    }
    if constexpr (K >= 3) {
      const uint16_t* t4 = o4_table<NG, K>() + bl * n4 * 3;
#pragma unroll
      for (int s = 0; s < n4; ++s) {
        const uint16_t r0 = t4[3 * s], r1 = t4[3 * s + 1], r2 = t4[3 * s + 2];
        const V4<T> GL = load_block<NG, T>(Gs, r0, H);
        const V4<T> GM = load_block<NG, T>(Gs, r1, H);
        const V4<T> GR = load_block<NG, T>(Gs, r2, H);
        o4_add(GL, GM, GR, (ref_neg(r0) ^ ref_neg(r1) ^ ref_neg(r2)) ? T(-1) : T(1), acc);
      }
    }
    const T inv = mt.ginv[mb];
    V4<T> g;
#pragma unroll
    for (int k = 0; k < 4; ++k) g.c[k] = inv * acc.c[k];
    gs_store<NG, T>(Gs, blk_off<NG>()[b] + c, g);
  }
}

// Shared memory of one warp: per event of the warp its gluon sub-currents
// G(B) and the 2^NG suffix momenta, and for every lane its colour-ordered
// amplitudes J[sigma][top helicity], kept in two planes (real, imaginary
// parts), each [row = sigma * 2 + top helicity][kJStride] with the lane as the
// column.  For FP32 the padded stride (36 = 4 mod 16 words) keeps both the
// lane-parallel stores and the tensor-core colour sum's fragment loads free of
// bank conflicts; the other types (no tensor-core path) use 32.
template <typename T> constexpr int kJStride = std::is_same<T, float>::value ? 36 : 32;
template <int NG, typename T> constexpr int kJPlane = TTNG<NG>::NPERM * 2 * kJStride<T>;
// The two-gluon suffix currents are shared through shared memory for plain
// FP32/FP64; the dual-number instantiations (derivative kernels) recompute
// them per lane, which keeps their (three times larger) shared footprint down.
template <typename T> constexpr bool kShareSuffixes = std::is_same<T, float>::value || std::is_same<T, double>::value;

template <int NG, typename T> struct WarpMem {
  static constexpr int EPW = Lanes<NG>::EPW;
  static constexpr size_t gs_bytes = sizeof(V4<T>) * EPW * TTNG<NG>::NSTORE;   // EPW component-major stores
  static constexpr size_t pt_off = gs_bytes;
  static constexpr size_t pt_bytes = MaskTab<NG, T>::bytes * EPW;       // EPW mask tables
  static constexpr size_t j_off = (pt_off + pt_bytes + 15) & ~size_t(15);
  static constexpr size_t j_bytes = sizeof(T) * 2 * kJPlane<NG, T>;
  // per event: the two-gluon suffix currents R(S), |S| = 2, for every ordered
  // pair, helicity pair and antitop helicity (component-major, NR2 each)
  static constexpr int NR2 = (NG >= 3 && kShareSuffixes<T>) ? NG * (NG - 1) * 8 : 0;
  static constexpr size_t r2_off = (j_off + j_bytes + 15) & ~size_t(15);
  static constexpr size_t r2_bytes = sizeof(cplx<T>) * 4 * NR2 * EPW;
  static constexpr size_t bytes = (r2_off + r2_bytes + 15) & ~size_t(15);
};

// Per-lane context of the quark-line walk.
template <typename T> struct LaneCtx {
  const cplx<T>* Gs;    // this event's sub-currents (component-major)
  const R4<T>* Ptab;    // -(q_tbar + sum of the gluon momenta in mask), by mask
  const cplx<T>* qf;    // heavy-quark propagator factor, by mask
  uint64_t pk;          // 4-bit compressed helicity index of this lane for every gluon mask
  S4<T> ub0, ub1;       // ubar(t) for top helicity -1, +1
  T m, mw;
  T* J;                 // &Jre[0][lane] of this warp (the imaginary plane follows at kJPlane)
  const cplx<T>* R2;    // this event's two-gluon suffix currents (component-major)
  unsigned ltb;         // antitop helicity bit of this lane
};

template <int NG, typename T>
__device__ __forceinline__ V4<T> lane_block(const LaneCtx<T>& cx, uint16_t ref) {
  const unsigned idx = unsigned(cx.pk >> (4 * ref_mask(ref))) & 15u;
  V4<T> g = gs_load<NG, T>(cx.Gs, ref_off(ref) + idx);
  if (ref_neg(ref)) g = neg(g);
  return g;
}

// Depth-first walk over the ordered suffixes S of the quark line (level LV =
// |S|): R(S) = -(P_S-slash + m)/(P_S^2 - m^2 + i m Gamma) sum_m G(S[:m])-slash R(S[m:]),
// then at the last level every completion sigma = (a,) + S gives
// J_sigma = ubar(t) sum_m G(sigma[:m])-slash R(sigma[m:]).  R[l] holds the
// current path's level-l current (R[0] = v(tbar)).  All lanes of a warp walk
// the same path (warp-uniform table reads), each with its own helicities.
template <int NG, int LV, typename T>
__device__ __forceinline__ void quark_walk(int parent, S4<T> (&R)[NG], const LaneCtx<T>& cx) {
  using PT = Paths<NG>;
  const int first = PT::template first<LV>(parent);
#pragma unroll (LV == NG - 1 ? 2 : 1)
  for (int k = 0; k <= NG - LV; ++k) {
    const int path = first + k;
    const uint8_t msk = PT::template mask<LV>(path);
    if constexpr (LV == 2 && kShareSuffixes<T>) {
      // computed once per event by the group (shared_suffixes)
      constexpr int NR2 = WarpMem<NG, T>::NR2;
      const int idx = path * 8 + int((unsigned(cx.pk >> (4 * msk)) & 15u) | (cx.ltb << 2));
#pragma unroll
      for (int c = 0; c < 4; ++c) R[2].c[c] = cx.R2[c * NR2 + idx];
    } else {
      S4<T> X = apply(make_slash(lane_block<NG, T>(cx, PT::template blk<LV>(path, 0))), R[LV - 1]);
#pragma unroll
      for (int m = 1; m < LV; ++m)
        apply_acc(make_slash(lane_block<NG, T>(cx, PT::template blk<LV>(path, m))), R[LV - 1 - m], X);
      R[LV] = quark_prop_f(cx.Ptab[msk], cx.m, cx.qf[msk], X);
    }
    if constexpr (LV < NG - 1) {
      quark_walk<NG, LV + 1, T>(path, R, cx);
    } else {
      S4<T> W = apply(make_slash(lane_block<NG, T>(cx, PT::final_blk(path, 0))), R[NG - 1]);
#pragma unroll
      for (int m = 1; m < NG; ++m)
        apply_acc(make_slash(lane_block<NG, T>(cx, PT::final_blk(path, m))), R[NG - 1 - m], W);
      const int sig = PT::final_sigma(path);
      const cplx<T> j0 = rowdot(cx.ub0, W), j1 = rowdot(cx.ub1, W);
      cx.J[(sig * 2 + 0) * kJStride<T>] = j0.r;
      cx.J[(sig * 2 + 0) * kJStride<T> + kJPlane<NG, T>] = j0.i;
      cx.J[(sig * 2 + 1) * kJStride<T>] = j1.r;
      cx.J[(sig * 2 + 1) * kJStride<T> + kJPlane<NG, T>] = j1.i;
    }
  }
}

// The two-gluon suffix currents R(S) = -(P_S-slash + m)/(P_S^2 - m^2 + i m Gamma)
// [G(S[:1])-slash R(S[1:]) + G(S)-slash v] depend on the helicities of two
// gluons and of the antitop only, so every lane of the group would compute
// each of them 2^(NG-2) times; the group computes each once (item = ordered
// pair, two gluon helicities, antitop helicity) and the lanes' walks read
// them.  Level-1 currents are recomputed per item.  Level-2 paths of one
// level-1 parent p1 are p1 (NG - 1) .. p1 (NG - 1) + NG - 2 (generator order).
template <int NG, typename T>
__device__ __forceinline__ void shared_suffixes(const cplx<T>* Gs, const MaskTab<NG, T>& mtab, const R4<T>& qtb, T mt,
                                                cplx<T>* R2, int gl) {
  using PT = Paths<NG>;
  constexpr int L = Lanes<NG>::L, NR2 = WarpMem<NG, T>::NR2;
  for (int it = gl; it < NR2; it += L) {
    const int p2 = it >> 3, sub = it & 7, p1 = p2 / (NG - 1);
    const unsigned m1 = PT::template mask<1>(p1), m2 = PT::template mask<2>(p2);
    const unsigned Hi = pdep_mask<NG>(unsigned(sub & 3), m2);
    const S4<T> v = v_out(qtb, mt, (sub & 4) ? 1 : -1);
    const uint16_t b1 = PT::template blk<1>(p1, 0), b20 = PT::template blk<2>(p2, 0), b21 = PT::template blk<2>(p2, 1);
    const S4<T> X1 = apply(make_slash(load_block<NG, T>(Gs, b1, Hi)), v);
    S4<T> R1 = quark_prop_f(mtab.ptab[m1], mt, mtab.qf[m1], X1);
    if (ref_neg(b1)) R1 = neg(R1);
    S4<T> X2 = apply(make_slash(load_block<NG, T>(Gs, b20, Hi)), R1);
    if (ref_neg(b20)) X2 = neg(X2);
    S4<T> Y = apply(make_slash(load_block<NG, T>(Gs, b21, Hi)), v);
    if (ref_neg(b21)) Y = neg(Y);
#pragma unroll
    for (int c = 0; c < 4; ++c) X2.c[c] = X2.c[c] + Y.c[c];
    const S4<T> R = quark_prop_f(mtab.ptab[m2], mt, mtab.qf[m2], X2);
#pragma unroll
    for (int c = 0; c < 4; ++c) R2[c * NR2 + it] = R.c[c];
  }
}

// ----------------------------------------------------------------------------
// Colour sum on the tensor cores (MF_FP32_TC).  The warp's amplitudes form
// B[sigma][n] with 128 columns n = (real/imaginary, top helicity, lane); the
// quadratic form of every column with C is Y = (D C) B followed by
// sum_sigma B[sigma][n] Y[sigma][n], and an event's |M|^2 sums the columns of
// its lanes.  Y comes from mma.m16n8k8 in TF32 with FP32 accumulation: the
// integer matrix D C (|entries| <= 2048) is exact in TF32, and B is split as
// B_hi + B_lo (both TF32), so Y = (D C) B_hi + (D C) B_lo carries ~22 bits of
// B.  Fragment layouts (PTX ISA, mma.m16n8k8 .tf32): A register r of lane l is
// (row l/4 + 8 (r & 1), column l%4 + 4 (r >> 1)); B register r is (row l%4 + 4 r,
// column l/4); accumulator register r is (row l/4 + 8 (r >> 1), column
// 2 (l%4) + (r & 1)).
__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// J^dagger (D C) J summed over the columns of each event of the warp; returns
// the sum of this lane's event (the value of group `group`).  J: the warp's
// real plane (the imaginary plane follows at kJPlane).  All 32 lanes call it.
template <int NG>
__device__ __forceinline__ float colour_sum_tc(const float* J, int group) {
  constexpr int NP = TTNG<NG>::NPERM, MT = ColourTC<NG>::MT, KS = ColourTC<NG>::KS;
  constexpr int L = Lanes<NG>::L, EPW = Lanes<NG>::EPW;
  const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  uint32_t a[MT][KS][4];
  const float* fa = colour_frag_a<NG>();
#pragma unroll
  for (int mi = 0; mi < MT; ++mi)
#pragma unroll
    for (int ks = 0; ks < KS; ++ks)
#pragma unroll
      for (int r = 0; r < 4; ++r) a[mi][ks][r] = __float_as_uint(__ldg(fa + ((mi * KS + ks) * 4 + r) * 32 + lane));
  float part[EPW];
#pragma unroll
  for (int e = 0; e < EPW; ++e) part[e] = 0.f;
#pragma unroll 1
  for (int u = 0; u < 4; ++u) {                 // u = 2 * (imaginary plane) + top helicity
    const float* P = J + (u >> 1) * kJPlane<NG, float>;
    const int h = u & 1;
#pragma unroll
    for (int c = 0; c < 4; ++c) {               // columns: lanes 8c .. 8c + 7
      const int lc0 = 8 * c;
      float d[MT][4];
#pragma unroll
      for (int mi = 0; mi < MT; ++mi)
#pragma unroll
        for (int r = 0; r < 4; ++r) d[mi][r] = 0.f;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        const int s0 = 8 * ks + tig, s1 = s0 + 4;
        const float x0 = s0 < NP ? P[(s0 * 2 + h) * kJStride<float> + lc0 + gid] : 0.f;
        const float x1 = s1 < NP ? P[(s1 * 2 + h) * kJStride<float> + lc0 + gid] : 0.f;
        const uint32_t h0 = tf32_bits(x0), h1 = tf32_bits(x1);
        const uint32_t l0 = tf32_bits(x0 - __uint_as_float(h0)), l1 = tf32_bits(x1 - __uint_as_float(h1));
#pragma unroll
        for (int mi = 0; mi < MT; ++mi) {
          mma_tf32(d[mi], a[mi][ks], h0, h1);
          mma_tf32(d[mi], a[mi][ks], l0, l1);
        }
      }
      float s = 0.f;
#pragma unroll
      for (int mi = 0; mi < MT; ++mi)
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          const int sg = 16 * mi + gid + 8 * hf;
          if (sg < NP) {
            const float2 b = *reinterpret_cast<const float2*>(P + (sg * 2 + h) * kJStride<float> + lc0 + 2 * tig);
            s = fmaf(d[mi][2 * hf], b.x, fmaf(d[mi][2 * hf + 1], b.y, s));
          }
        }
      part[lc0 / L] += s;
    }
  }
  float mine = 0.f;
#pragma unroll
  for (int e = 0; e < EPW; ++e) {
    float v = part[e];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (e == group) mine = v;
  }
  return mine;
}

// The last level of the quark line for one completion: J_sigma for both top
// helicities of the level-(NG-1) path `path`, R[l] the path's level-l currents.
template <int NG, typename T>
__device__ __forceinline__ void final_amplitudes(int path, const S4<T> (&R)[NG], const LaneCtx<T>& cx) {
  using PT = Paths<NG>;
  S4<T> W = apply(make_slash(lane_block<NG, T>(cx, PT::final_blk(path, 0))), R[NG - 1]);
#pragma unroll
  for (int m = 1; m < NG; ++m)
    apply_acc(make_slash(lane_block<NG, T>(cx, PT::final_blk(path, m))), R[NG - 1 - m], W);
  const int sig = PT::final_sigma(path);
  const cplx<T> j0 = rowdot(cx.ub0, W), j1 = rowdot(cx.ub1, W);
  cx.J[(sig * 2 + 0) * kJStride<T>] = j0.r;
  cx.J[(sig * 2 + 0) * kJStride<T> + kJPlane<NG, T>] = j0.i;
  cx.J[(sig * 2 + 1) * kJStride<T>] = j1.r;
  cx.J[(sig * 2 + 1) * kJStride<T> + kJPlane<NG, T>] = j1.i;
}

// The quark line of four gluons with the three-gluon currents shared by lane
// pairs.  R(S) for S = (a, b, c) does not depend on the helicity of the gluon g
// missing from S, so lanes l and l ^ (1 << g) need the same R(S) for both
// paths (a, b, c) and (b, a, c): each computes one, the partner's arrives by a
// shuffle.  Order: last gluon c (its level-1 current in registers), then the
// missing gluon g; the two-gluon currents come from the shared store.
template <typename T>
__device__ __forceinline__ void quark_walk_paired4(const S4<T>& v, const LaneCtx<T>& cx, unsigned H) {
  using PT = Paths<4>;
  constexpr int NR2 = WarpMem<4, T>::NR2;
  auto load_r2 = [&](int p2) {
    const uint8_t m2 = PT::template mask<2>(p2);
    const int idx = p2 * 8 + int((unsigned(cx.pk >> (4 * m2)) & 15u) | (cx.ltb << 2));
    S4<T> r;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.c[k] = cx.R2[k * NR2 + idx];
    return r;
  };
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
    S4<T> R[4];
    R[0] = v;
    const uint8_t m1 = PT::template mask<1>(c);
    R[1] = quark_prop_f(cx.Ptab[m1], cx.m, cx.qf[m1],
                        apply(make_slash(lane_block<4, T>(cx, PT::template blk<1>(c, 0))), v));
#pragma unroll 1
    for (int gi = 0; gi < 3; ++gi) {
      const int g = kL3Miss4[c * 3 + gi];
      const unsigned bit = (H >> g) & 1u;
      const int mine = kL3Pair4[(c * 3 + gi) * 2 + bit], other = kL3Pair4[(c * 3 + gi) * 2 + (bit ^ 1u)];
      R[2] = load_r2(mine >> 1);
      S4<T> X = apply(make_slash(lane_block<4, T>(cx, PT::template blk<3>(mine, 0))), R[2]);
      apply_acc(make_slash(lane_block<4, T>(cx, PT::template blk<3>(mine, 1))), R[1], X);
      apply_acc(make_slash(lane_block<4, T>(cx, PT::template blk<3>(mine, 2))), v, X);
      const uint8_t m3 = PT::template mask<3>(mine);
      R[3] = quark_prop_f(cx.Ptab[m3], cx.m, cx.qf[m3], X);
      S4<T> Ro;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        Ro.c[k].r = __shfl_xor_sync(0xffffffffu, R[3].c[k].r, 1 << g);
        Ro.c[k].i = __shfl_xor_sync(0xffffffffu, R[3].c[k].i, 1 << g);
      }
      final_amplitudes<4, T>(mine, R, cx);
      R[2] = load_r2(other >> 1);
      R[3] = Ro;
      final_amplitudes<4, T>(other, R, cx);
    }
  }
}

// One entry of the mask table of an event (helicity independent): for the
// gluon subset `msk`, the momentum sum K (incoming gluons negated), -(q_tbar +
// K), 1/K^2 (two or more gluons) and the top-propagator factor.  q: the
// gluons' outgoing-convention momenta, qtb: the antitop's.
template <int NG, typename T>
__device__ __forceinline__ void mask_entry(const R4<T> (&q)[NG], const R4<T>& qtb, int msk, const MaskTab<NG, T>& mtab,
                                           T mt, T mw) {
  R4<T> K = {{T(0), T(0), T(0), T(0)}};
#pragma unroll
  for (int g = 0; g < NG; ++g)
    if ((msk >> g) & 1) K = K + q[g];
  const R4<T> P = qtb + K;
  mtab.qsum[msk] = K;
  mtab.ptab[msk] = -P;
  const T k2 = mdot(K, K);
  T den = mdot(P, P) - mt * mt;
  if constexpr (sizeof(value_of(T(0))) == sizeof(float)) {
    // FP32, subsets of outgoing gluons only (the top propagator that can come
    // near its pole, t -> t + soft or collinear g): with massless gluons and
    // an on-shell antitop, P^2 - m^2 = 2 q_tbar.K + sum_{i<j} 2 q_i.q_j, a sum
    // of non-negative terms, free of the cancellation of P^2 against m^2
    // that costs ~E^2/|P^2 - m^2| ulps.  With an incoming gluon the terms
    // have both signs and the direct form is kept.
    if ((msk & 3) == 0) {
      T pairs = T(0);
#pragma unroll
      for (int i = 2; i < NG; ++i)
#pragma unroll
        for (int j = i + 1; j < NG; ++j)
          if (((msk >> i) & 1) && ((msk >> j) & 1)) pairs += T(2) * mdot(q[i], q[j]);
      den = fma(T(2), mdot(qtb, K), pairs);
    }
  }
  mtab.ginv[msk] = __popc(unsigned(msk)) >= 2 ? T(1) / k2 : T(0);
  const T inv = T(-1) / fma(den, den, mw * mw);
  mtab.qf[msk] = {den * inv, -mw * inv};     // -1/den = -conj(den)/|den|^2
}

// The gluons' outgoing-convention momenta (incoming ones negated) of an event
// given in MadGraph order (legs 0, 1 incoming gluons, 2 top, 3 antitop, then
// the final gluons).
template <int NG, typename T>
__device__ __forceinline__ void gluon_momenta(const T (&p)[NG + 2][4], R4<T> (&q)[NG]) {
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const int leg = g < 2 ? g : g + 2;
    const T s = g < 2 ? T(-1) : T(1);
#pragma unroll
    for (int c = 0; c < 4; ++c) q[g].v[c] = s * p[leg][c];
  }
}

// The four-gluon quark line in FP32 with both antitop helicities of a gluon
// helicity pattern H in one lane, as packed pairs (f2: half 0 = antitop
// helicity -1, half 1 = +1), each lane taking the last gluons c of its half of
// the warp (lanes 0-15: c = 0, 1; lanes 16-31: c = 2, 3).  The suffix
// currents depend on the antitop helicity through v(tbar) only, so the two
// halves run the same walk on different data and every FP32 operation of
// the walk issues once for both.  Lane H + 16 h computes what lane H + 16 h
// of quark_walk_paired4 would for its c (the same three-gluon pairing
// between lanes l and l ^ 2^g, now within a half), and the amplitudes land
// in the same columns of the J planes (column H + 16 (antitop bit)), so
// the colour sums that follow are unchanged.  Results equal the scalar
// walk's: each half of a paired instruction rounds as the scalar one.
__device__ __forceinline__ void final_amplitudes_x2(int path, const S4<f2> (&R)[4], const LaneCtx<float>& cx,
                                                    float* J0, float* J1) {
  using PT = Paths<4>;
  // two independent partial sums (the paired instructions' latency is longer
  // than the scalar ones', so shorter dependency chains keep them issuing)
  S4<f2> W = apply(dup(make_slash(lane_block<4, float>(cx, PT::final_blk(path, 0)))), R[3]);
  S4<f2> V = apply(dup(make_slash(lane_block<4, float>(cx, PT::final_blk(path, 2)))), R[1]);
  apply_acc(dup(make_slash(lane_block<4, float>(cx, PT::final_blk(path, 1)))), R[2], W);
  apply_acc(dup(make_slash(lane_block<4, float>(cx, PT::final_blk(path, 3)))), R[0], V);
#pragma unroll
  for (int k = 0; k < 4; ++k) W.c[k] = W.c[k] + V.c[k];
  const int sig = PT::final_sigma(path);
  const cplx<f2> j0 = rowdot(cx.ub0, W), j1 = rowdot(cx.ub1, W);
  constexpr int S = kJStride<float>, P = kJPlane<4, float>;
  J0[(sig * 2 + 0) * S] = j0.r.v.x;
  J0[(sig * 2 + 0) * S + P] = j0.i.v.x;
  J0[(sig * 2 + 1) * S] = j1.r.v.x;
  J0[(sig * 2 + 1) * S + P] = j1.i.v.x;
  J1[(sig * 2 + 0) * S] = j0.r.v.y;
  J1[(sig * 2 + 0) * S + P] = j0.i.v.y;
  J1[(sig * 2 + 1) * S] = j1.r.v.y;
  J1[(sig * 2 + 1) * S + P] = j1.i.v.y;
}

__device__ __forceinline__ void quark_walk_paired4_x2(const S4<f2>& v, const LaneCtx<float>& cx, unsigned H,
                                                      int half, float* J0, float* J1) {
  using PT = Paths<4>;
  constexpr int NR2 = WarpMem<4, float>::NR2;
  auto load_r2 = [&](int p2) {
    const uint8_t m2 = PT::template mask<2>(p2);
    const int idx = p2 * 8 + int(unsigned(cx.pk >> (4 * m2)) & 15u);
    S4<f2> r;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.c[k] = pack(cx.R2[k * NR2 + idx], cx.R2[k * NR2 + idx + 4]);
    return r;
  };
#pragma unroll 1
  for (int ci = 0; ci < 2; ++ci) {
    const int c = 2 * half + ci;
    S4<f2> R[4];
    R[0] = v;
    const uint8_t m1 = PT::template mask<1>(c);
    R[1] = quark_prop_f(dup(cx.Ptab[m1]), f2(cx.m), dup(cx.qf[m1]),
                        apply(dup(make_slash(lane_block<4, float>(cx, PT::template blk<1>(c, 0)))), v));
#pragma unroll 1
    for (int gi = 0; gi < 3; ++gi) {
      const int g = kL3Miss4[c * 3 + gi];
      const unsigned bit = (H >> g) & 1u;
      const int mine = kL3Pair4[(c * 3 + gi) * 2 + bit], other = kL3Pair4[(c * 3 + gi) * 2 + (bit ^ 1u)];
      R[2] = load_r2(mine >> 1);
      S4<f2> X = apply(dup(make_slash(lane_block<4, float>(cx, PT::template blk<3>(mine, 0)))), R[2]);
      apply_acc(dup(make_slash(lane_block<4, float>(cx, PT::template blk<3>(mine, 1)))), R[1], X);
      apply_acc(dup(make_slash(lane_block<4, float>(cx, PT::template blk<3>(mine, 2)))), v, X);
      const uint8_t m3 = PT::template mask<3>(mine);
      R[3] = quark_prop_f(dup(cx.Ptab[m3]), f2(cx.m), dup(cx.qf[m3]), X);
      S4<f2> Ro;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        Ro.c[k].r.v.x = __shfl_xor_sync(0xffffffffu, R[3].c[k].r.v.x, 1 << g);
        Ro.c[k].r.v.y = __shfl_xor_sync(0xffffffffu, R[3].c[k].r.v.y, 1 << g);
        Ro.c[k].i.v.x = __shfl_xor_sync(0xffffffffu, R[3].c[k].i.v.x, 1 << g);
        Ro.c[k].i.v.y = __shfl_xor_sync(0xffffffffu, R[3].c[k].i.v.y, 1 << g);
      }
      // the two completions in one loop body: the packed code is about twice
      // the scalar walk's per instruction issued, and two inlined copies of
      // the last level overflow the instruction cache
      int path = mine;
#pragma unroll 1
      for (int w = 0; w < 2; ++w) {
        final_amplitudes_x2(path, R, cx, J0, J1);
        if (w == 0) {
          R[2] = load_r2(other >> 1);
          R[3] = Ro;
          path = other;
        }
      }
    }
  }
}

// Per event, helicity independent: the mask table (one subset per lane, see
// mask_entry) and the polarisation vectors (level-1 sub-currents).
template <int NG, typename T>
__device__ __forceinline__ void event_tables(const T (&p)[NG + 2][4], const MaskTab<NG, T>& mtab, cplx<T>* Gs, int gl,
                                             T mt, T mw) {
  constexpr int L = Lanes<NG>::L;
  R4<T> q[NG];
  gluon_momenta<NG, T>(p, q);
  R4<T> qtb;
#pragma unroll
  for (int c = 0; c < 4; ++c) qtb.v[c] = p[3][c];
  if (gl < (1 << NG)) mask_entry<NG, T>(q, qtb, gl, mtab, mt, mw);
  for (int it = gl; it < 2 * NG; it += L) {
    const int g = it >> 1;
    const int leg = g < 2 ? g : g + 2;
    R4<T> k;
#pragma unroll
    for (int c = 0; c < 4; ++c) k.v[c] = p[leg][c];
    gs_store<NG, T>(Gs, 2 * g + (it & 1), polarisation(k, (it & 1) ? 1 : -1, g >= 2));
  }
}

// |M|^2 (without the normalisation MeParams::norm) of one event, computed by
// its lane group; p: physical momenta in MadGraph order; wm: this warp's
// shared memory (WarpMem layout); tc: colour sum on the tensor cores (FP32
// only).  Every lane of the warp must call this (the group synchronises with
// __syncwarp).
template <int NG, typename T>
__device__ __forceinline__ T group_me2(const T (&p)[NG + 2][4], unsigned char* wm, int group, int gl, T mt, T mw,
                                       int tc = 0) {
  using WM = WarpMem<NG, T>;
  constexpr int L = Lanes<NG>::L;
  constexpr int NP = TTNG<NG>::NPERM;
  cplx<T>* Gs = reinterpret_cast<cplx<T>*>(wm) + group * 4 * TTNG<NG>::NSTORE;
  const MaskTab<NG, T> mtab(wm + WM::pt_off + group * MaskTab<NG, T>::bytes);
  T* Jw = reinterpret_cast<T*>(wm + WM::j_off);
  cplx<T>* R2 = reinterpret_cast<cplx<T>*>(wm + WM::r2_off) + group * 4 * WM::NR2;
  const int lane = threadIdx.x & 31;
  R4<T> qtb, pt;
#pragma unroll
  for (int c = 0; c < 4; ++c) { qtb.v[c] = p[3][c]; pt.v[c] = p[2][c]; }
  event_tables<NG, T>(p, mtab, Gs, gl, mt, mw);
  __syncwarp();
  gluon_level<NG, 2, T>(mtab, Gs, gl);
  if constexpr (NG >= 3) { __syncwarp(); gluon_level<NG, 3, T>(mtab, Gs, gl); }
  if constexpr (NG >= 4) { __syncwarp(); gluon_level<NG, 4, T>(mtab, Gs, gl); }
  __syncwarp();
  if constexpr (NG >= 3 && kShareSuffixes<T>) {
    shared_suffixes<NG, T>(Gs, mtab, qtb, mt, R2, gl);
    __syncwarp();
  }
  // quark line of this lane
  const unsigned H = unsigned(gl) & ((1u << NG) - 1u);
  const int ltb = ((gl >> NG) & 1) ? 1 : -1;
  LaneCtx<T> cx;
  cx.Gs = Gs;
  cx.Ptab = mtab.ptab;
  cx.qf = mtab.qf;
  cx.pk = 0;
#pragma unroll
  for (unsigned msk = 1; msk < (1u << NG); ++msk) cx.pk |= uint64_t(pext_mask<NG>(H, msk)) << (4 * msk);
  cx.ub0 = ubar_out(pt, mt, -1);
  cx.ub1 = ubar_out(pt, mt, 1);
  cx.m = mt;
  cx.mw = mw;
  cx.J = Jw + lane;
  cx.R2 = R2;
  cx.ltb = unsigned((gl >> NG) & 1);
  S4<T> R[NG];
  R[0] = v_out(qtb, mt, ltb);
  if constexpr (NG == 4 && std::is_same<T, float>::value && kPackedWalk) {
    // both antitop helicities of pattern H in this lane, packed; c by warp half
    quark_walk_paired4_x2(pack(v_out(qtb, mt, -1), v_out(qtb, mt, 1)), cx, H, gl >> 4, Jw + H, Jw + H + 16);
    __syncwarp();   // every column of this lane's colour sum was written by the lanes of both halves
  } else if constexpr (NG == 4 && kShareSuffixes<T>) {
    quark_walk_paired4<T>(R[0], cx, H);
  } else {
    quark_walk<NG, 1, T>(0, R, cx);
  }
  if constexpr (std::is_same<T, float>::value) {
    if (tc) {
      __syncwarp();   // every lane's J is in shared memory
      const float v = colour_sum_tc<NG>(Jw, group);
      __syncwarp();   // the warp's shared store may be overwritten after this
      return v;
    }
  }
  // colour sum of both top helicities from this lane's amplitudes
  T part = T(0);
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    cplx<T> J[NP];
#pragma unroll
    for (int sg = 0; sg < NP; ++sg)
      J[sg] = {cx.J[(sg * 2 + h) * kJStride<T>], cx.J[(sg * 2 + h) * kJStride<T> + kJPlane<NG, T>]};
    part += colour_form<T>(J);
  }
#pragma unroll
  for (int off = L / 2; off > 0; off >>= 1) part += shfl_xor_any(0xffffffffu, part, off);
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
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int group = lane / L, gl = lane % L;
  unsigned char* wm = smem_raw + warp * WarpMem<NG, T>::bytes;
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
    const T v = group_me2<NG, T>(p, wm, group, gl, mt, mw, mp.colour_tc);
    if (ok && gl == 0) out[e] = double(v) * mp.norm;
  }
}

// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_sample(SampleParams sp, const double* __restrict__ edges_g, int64_t n,
                                                     uint64_t seed, int iter, double* __restrict__ mom,
                                                     double* __restrict__ wps, uint8_t* __restrict__ bins);

// Vegas accumulators of one CTA: [0] sum w, [1] sum w^2, [2 + j*nbins + b] sum w^2 in bin b of dim j
__device__ __forceinline__ void accumulate_event(double w, const uint8_t (&b_ev)[kMaxDim], int ndim, int nbins,
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
#pragma unroll 1
  for (int j = 0; j < ndim; ++j) {
    const unsigned b = b_ev[j];
    // lanes holding the same bin form a group; reduce it with a shuffle tree
    // (rank r adds rank r + s for s = 1, 2, 4, ...; rank 0 holds the sum)
    const unsigned peers = __match_any_sync(full, b);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const unsigned above = peers & ~((2u << lane) - 1u);
    double v = w2;
#pragma unroll 1
    for (int s = 1; s < 32; s <<= 1) {
      unsigned m = above;
#pragma unroll 1
      for (int k = 1; k < s && m; ++k) m &= m - 1u;
      const int src = m ? (__ffs(m) - 1) : lane;
      const double o = __shfl_sync(full, v, src);
      if (m && (rank % (2 * s)) == 0) v += o;
    }
    if (rank == 0) atomicAdd(&hist[j * nbins + b], v);
  }
}

// Shared-memory layout of k_fused (bytes), shared by host and device: the
// CTA's grid edges and Vegas sums, then one WarpMem per warp.
template <int NG, typename T> struct FusedLayout {
  __host__ __device__ static size_t al(size_t x) { return (x + 15) & ~size_t(15); }
  __host__ __device__ static size_t edges(int, int) { return 0; }
  __host__ __device__ static size_t hist(int ndim, int nbins) { return al(edges(ndim, nbins) + sizeof(double) * ndim * (nbins + 1)); }
  __host__ __device__ static size_t sums(int ndim, int nbins) { return al(hist(ndim, nbins) + sizeof(double) * ndim * nbins); }
  __host__ __device__ static size_t warps(int ndim, int nbins) { return al(sums(ndim, nbins) + sizeof(double) * 2); }
  __host__ __device__ static size_t total(int ndim, int nbins) {
    return al(warps(ndim, nbins) + WarpMem<NG, T>::bytes * kWarps);
  }
};

// Persistent fused kernel; every warp works on its own blocks of 32 events:
//   phase 1 (lane per event): Philox -> Vegas -> luminosity -> RAMBO -> cuts;
//   phase 2 (lane group per event that passed): |M|^2, the event's momenta
//     broadcast from its lane with shuffles;
//   phase 3 (lane per event): w = |M|^2 * prefactor, Vegas sums.
// No block-wide barrier inside the event loop.  partials[blockIdx.x * nacc + k]
// receives the CTA's sums (nacc = 2 + ndim*nbins); counters[blockIdx.x * 2 + {0,1}]
// = events passing cuts, Newton misses.  Weights (if w_out) are indexed by the
// event's position 0..n-1 in this call; the Philox counter is first_event + position.
template <int NG, typename T>
__global__ void __launch_bounds__(kThreads, 2) k_fused(SampleParams sp, MeParams mp, const double* __restrict__ edges_g,
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
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int group = lane / L, gl = lane % L;
  unsigned char* wm = smem_raw + LY::warps(ndim, nbins) + warp * WarpMem<NG, T>::bytes;
  for (int i = t; i < ndim * (nbins + 1); i += kThreads) edges[i] = edges_g[i];
  for (int i = t; i < ndim * nbins; i += kThreads) hist[i] = 0.0;
  if (t < 2) sums[t] = 0.0;
  unsigned long long npass = 0, nfail = 0;
  const T mt = T(mp.mt), mw = T(mp.mw);
  const unsigned full = 0xffffffffu;
  __syncthreads();

  const int64_t stride = int64_t(gridDim.x) * kWarps * 32;
  for (int64_t base = (int64_t(blockIdx.x) * kWarps + warp) * 32; base < n; base += stride) {
    const int64_t ev = base + lane;
    const bool valid = ev < n;
    EventKin<T> k;
    k.prefactor = 0.0;
    k.pass = 0;
    if (valid) {
      sample_event(sp, edges, seed, iter, uint64_t(first_event + ev), k);
      npass += k.pass;
      nfail += k.newton_fail;
    } else {
      for (int j = 0; j < kMaxDim; ++j) k.bins[j] = 0;
    }
    T mine[NEXT][4];
#pragma unroll
    for (int i = 0; i < NEXT; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) mine[i][c] = k.p[i][c];
    double me = 0.0;
    unsigned todo = __ballot_sync(full, valid && k.pass);
    while (todo) {
      // the next EPW events that passed: group g takes the g-th lowest set bit
      int src = -1;
      unsigned rest = todo;
#pragma unroll
      for (int g = 0; g < EPW; ++g) {
        const int b = rest ? __ffs(rest) - 1 : -1;
        if (g == group) src = b;
        if (rest) rest &= rest - 1u;
      }
      const int from = src < 0 ? 0 : src;
      T p[NEXT][4];
#pragma unroll
      for (int i = 0; i < NEXT; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) p[i][c] = __shfl_sync(full, mine[i][c], from);
      const T v = group_me2<NG, T>(p, wm, group, gl, mt, mw, mp.colour_tc);
#pragma unroll
      for (int g = 0; g < EPW; ++g) {
        const T vg = __shfl_sync(full, v, g * L);
        const int sg = __shfl_sync(full, src, g * L);
        if (sg == lane) me = double(vg) * mp.norm;
      }
      todo = rest;
    }
    const double w = valid ? me * k.prefactor : 0.0;
    if (w_out != nullptr && valid) w_out[ev] = w;
    accumulate_event(w, k.bins, ndim, nbins, sums, hist);
  }
  __syncthreads();
  const int nacc = 2 + ndim * nbins;
  double* dst = partials + int64_t(blockIdx.x) * nacc;
  for (int i = t; i < ndim * nbins; i += kThreads) dst[2 + i] = hist[i];
  if (t < 2) dst[t] = sums[t];
  // CTA totals of the counters
  for (int off = 16; off > 0; off >>= 1) {
    npass += __shfl_xor_sync(full, npass, off);
    nfail += __shfl_xor_sync(full, nfail, off);
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

// ----------------------------------------------------------------------------
// Two-kernel iteration: k_sample_rec writes one compact record per event
// (coalesced, SoA) and the list of events that passed the cuts; k_me_acc
// walks that list with one lane group per event, like k_matrix_element,
// evaluates |M|^2 and accumulates the Vegas sums (events that failed add 0 to
// every sum).  Splitting the sampling (a long, branchy FP64/transcendental
// code path) from the amplitude loop keeps the amplitude kernel's instruction
// working set small and its warps in step; the records cost ~2 x 90 bytes of
// HBM traffic per event, negligible next to ~1 MFLOP of amplitude work.
//
// Record layout for a chunk of C events (K = kinematics type):
//   mom  [n_final*4][C] K    final-state momenta (t, tbar, gluons), components E, px, py, pz
//   rs   [C]            K    partonic sqrt(s_hat) (the beams are (rs/2)(1, 0, 0, +-1))
//   pref [C]            f64  weight without |M|^2
//   flag [ndim][C]      u8   Vegas bin of each dimension
//   list [C]            i32  positions of the events that passed (first *count entries)
//   count[2]            u32  events that passed, Newton misses
template <typename K> struct RecordView {
  K* mom;
  K* rs;
  double* pref;
  uint8_t* flag;
  int* list;
  unsigned* count;
  int64_t C;
  __host__ __device__ static size_t al(size_t x) { return (x + 255) & ~size_t(255); }
  __host__ __device__ static size_t bytes(int n_final, int ndim, int64_t C) {
    size_t o = al((size_t(n_final) * 4 + 1) * sizeof(K) * C);
    o = al(o + sizeof(double) * C);
    o = al(o + size_t(ndim) * C);
    o = al(o + sizeof(int) * C);
    return o + 2 * sizeof(unsigned);
  }
  __host__ __device__ static RecordView carve(void* base, int n_final, int ndim, int64_t C) {
    RecordView v;
    unsigned char* p = static_cast<unsigned char*>(base);
    v.C = C;
    v.mom = reinterpret_cast<K*>(p);
    v.rs = v.mom + size_t(n_final) * 4 * C;
    size_t o = al((size_t(n_final) * 4 + 1) * sizeof(K) * C);
    v.pref = reinterpret_cast<double*>(p + o);
    o = al(o + sizeof(double) * C);
    v.flag = p + o;
    o = al(o + size_t(ndim) * C);
    v.list = reinterpret_cast<int*>(p + o);
    o = al(o + sizeof(int) * C);
    v.count = reinterpret_cast<unsigned*>(p + o);
    return v;
  }
};

// rec.count must be zero on entry.  Weights of the events that failed are
// written here (0); k_me_acc writes the others.
template <typename K>
__global__ void __launch_bounds__(kThreads) k_sample_rec(SampleParams sp, const double* __restrict__ edges_g,
                                                         int64_t first_event, int64_t n, uint64_t seed, int iter,
                                                         RecordView<K> rec, double* __restrict__ w_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* edges = reinterpret_cast<double*>(smem_raw);
  for (int i = threadIdx.x; i < sp.ndim * (sp.nbins + 1); i += blockDim.x) edges[i] = edges_g[i];
  __syncthreads();
  const int nf = sp.n_final;
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < n; base += stride) {
    const int64_t e = base + threadIdx.x;
    int pass = 0, fail = 0;
    if (e < n) {
      EventKin<K> k;
      sample_event(sp, edges, seed, iter, uint64_t(first_event + e), k);
#pragma unroll
      for (int i = 0; i < kMaxExt - 2; ++i)
        if (i < nf)
#pragma unroll
          for (int c = 0; c < 4; ++c) rec.mom[int64_t(i * 4 + c) * rec.C + e] = k.p[2 + i][c];
      rec.rs[e] = k.p[0][0] + k.p[1][0];
      rec.pref[e] = k.prefactor;
#pragma unroll
      for (int j = 0; j < kMaxDim; ++j)
        if (j < sp.ndim) rec.flag[int64_t(j) * rec.C + e] = k.bins[j];
      pass = k.pass;
      fail = k.newton_fail;
      if (!pass && w_out != nullptr) w_out[e] = 0.0;
    }
    const unsigned bal = __ballot_sync(full, pass);
    const unsigned fbal = __ballot_sync(full, fail);
    unsigned pos = 0;
    if (lane == 0) {
      if (bal) pos = atomicAdd(&rec.count[0], unsigned(__popc(bal)));
      if (fbal) atomicAdd(&rec.count[1], unsigned(__popc(fbal)));
    }
    pos = __shfl_sync(full, pos, 0);
    if (pass) rec.list[pos + __popc(bal & ((1u << lane) - 1u))] = int(e);
  }
}

// W: warps per CTA (the launch shape; 4 by default)
template <int NG, typename T, int W = kWarps> struct MeAccLayout {
  __host__ __device__ static size_t al(size_t x) { return (x + 15) & ~size_t(15); }
  __host__ __device__ static size_t hist(int) { return 0; }
  __host__ __device__ static size_t sums(int nacc) { return al(sizeof(double) * (nacc - 2)); }
  __host__ __device__ static size_t warps(int nacc) { return al(sums(nacc) + sizeof(double) * 2); }
  __host__ __device__ static size_t total(int nacc) { return al(warps(nacc) + WarpMem<NG, T>::bytes * W); }
};

// |M|^2 of the listed events, weights, Vegas sums.  partials[blockIdx.x * nacc + k]
// receive (accumulate = 0) or add (accumulate = 1) the CTA's sums; block 0
// also carries the chunk's counters.  W warps per CTA (32 W threads).
template <int NG, typename T, int W = kWarps>
__global__ void __launch_bounds__(32 * W, (8 / W) > 0 ? 8 / W : 1)
    k_me_acc(MeParams mp, int ndim, int nbins, RecordView<T> rec, int accumulate, double* __restrict__ partials,
             unsigned long long* __restrict__ counters, double* __restrict__ w_out) {
  using LY = MeAccLayout<NG, T, W>;
  constexpr int kThr = 32 * W;
  constexpr int EPW = Lanes<NG>::EPW, L = Lanes<NG>::L, NEXT = Lanes<NG>::NEXT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nacc = 2 + ndim * nbins;
  double* hist = reinterpret_cast<double*>(smem_raw + LY::hist(nacc));
  double* sums = reinterpret_cast<double*>(smem_raw + LY::sums(nacc));
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int group = lane / L, gl = lane % L;
  unsigned char* wm = smem_raw + LY::warps(nacc) + warp * WarpMem<NG, T>::bytes;
  for (int i = t; i < ndim * nbins; i += kThr) hist[i] = 0.0;
  if (t < 2) sums[t] = 0.0;
  const T mt = T(mp.mt), mw = T(mp.mw);
  const unsigned full = 0xffffffffu;
  const int64_t npass = rec.count[0];
  double s1 = 0.0, s2 = 0.0;
  __syncthreads();

  const int64_t stride = int64_t(gridDim.x) * W * EPW;
  for (int64_t base = (int64_t(blockIdx.x) * W + warp) * EPW; base < npass; base += stride) {
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
    const T v = group_me2<NG, T>(p, wm, group, gl, mt, mw, mp.colour_tc);
    if (ok) {
      const double w = double(v) * mp.norm * rec.pref[e];
      if (gl == 0) {
        s1 += w;
        s2 += w * w;
        if (w_out != nullptr) w_out[e] = w;
      }
      if (gl < ndim) atomicAdd(&hist[gl * nbins + rec.flag[int64_t(gl) * rec.C + e]], w * w);
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
  for (int i = t; i < ndim * nbins; i += kThr) dst[2 + i] = (accumulate ? dst[2 + i] : 0.0) + hist[i];
  if (t < 2) dst[t] = (accumulate ? dst[t] : 0.0) + sums[t];
  if (t < 2) {
    const unsigned long long c = blockIdx.x == 0 ? (unsigned long long)rec.count[t] : 0ull;
    counters[blockIdx.x * 2 + t] = (accumulate ? counters[blockIdx.x * 2 + t] : 0ull) + c;
  }
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
// |M|^2 + accumulation of records already sampled (rec_base: RecordView of capacity C)
template <int NG>
cudaError_t launch_me_acc(int precision, const MeParams& mp, int n_final, int ndim, int nbins, void* rec_base,
                          int64_t C, int accumulate, double* partials, unsigned long long* counters, double* w_out,
                          int grid, cudaStream_t s);
// two-kernel iteration over one chunk of records (rec_base: RecordView of chunk capacity C);
// me_warps > 0 selects the |M|^2 kernel with that many warps per CTA (g g -> t t~ g g, FP32 only)
template <int NG>
cudaError_t launch_chunk(int precision, const SampleParams& sp, const MeParams& mp, const double* edges,
                         int64_t first_event, int64_t n, int64_t C, void* rec_base, uint64_t seed, int iter,
                         int accumulate, double* partials, unsigned long long* counters, double* w_out, int grid,
                         cudaStream_t s, cudaEvent_t* ev = nullptr, int me_warps = 0);
// The FP32 g g -> t t~ g g |M|^2-and-accumulate kernel with `warps` (1..8) warps per
// CTA (mf_launch_shape.cu): its shared memory and occupancy, and a launch over
// the records of one chunk.
cudaError_t me_acc_shape_config(int warps, int ndim, int nbins, size_t* smem, int* ctas);
cudaError_t launch_me_acc_shape(int warps, const MeParams& mp, int n_final, int ndim, int nbins, void* rec_base,
                                int64_t C, int accumulate, double* partials, unsigned long long* counters,
                                double* w_out, int grid, cudaStream_t s);
template <int NG>
cudaError_t me_acc_config(int precision, int ndim, int nbins, size_t* smem, int* ctas_per_sm);
size_t record_bytes(int precision, int n_final, int ndim, int64_t C);
template <int NG>
cudaError_t me_config(int precision, size_t* smem, int* ctas_per_sm);

cudaError_t launch_sample(const SampleParams& sp, const double* edges, int64_t n, uint64_t seed, int iter,
                          double* mom, double* wps, uint8_t* bins, cudaStream_t s);
cudaError_t launch_uniforms(uint64_t seed, int iter, int64_t first_event, int64_t n, int ndim, double* y,
                            cudaStream_t s);
// hit-or-miss unweighting of one chunk of evaluated records (weights w[n])
cudaError_t launch_unweight(int precision, void* rec_base, int n_final, int ndim, int64_t C, const double* w,
                            int64_t n, uint64_t seed, int iter, int64_t first_event, double w_max, int64_t cap,
                            double* mom_out, double* weight_out, int64_t* event_out, unsigned long long* counts,
                            cudaStream_t s);
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
      *smem = WarpMem<NG, double>::bytes * kWarps;                                    \
      e = cudaFuncSetAttribute(k_matrix_element<NG, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem)); \
      if (e != cudaSuccess) return e;                                                                             \
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_matrix_element<NG, double>, kThreads, *smem);  \
    }                                                                                                             \
    *smem = WarpMem<NG, float>::bytes * kWarps;                                       \
    e = cudaFuncSetAttribute(k_matrix_element<NG, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem)); \
    if (e != cudaSuccess) return e;                                                                               \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_matrix_element<NG, float>, kThreads, *smem);     \
  }                                                                                                               \
  template <>                                                                                                     \
  cudaError_t launch_matrix_element<NG>(int precision, const MeParams& mp, int64_t n, const double* mom,          \
                                        double* out, int grid, cudaStream_t s) {                                  \
    if (precision == 0) {                                                                                         \
      const size_t sm = WarpMem<NG, double>::bytes * kWarps;                          \
      k_matrix_element<NG, double><<<grid, kThreads, sm, s>>>(mp, n, mom, out);                                   \
    } else {                                                                                                      \
      const size_t sm = WarpMem<NG, float>::bytes * kWarps;                           \
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
  cudaError_t me_acc_config<NG>(int precision, int ndim, int nbins, size_t* smem, int* ctas) {                    \
    cudaError_t e;                                                                                                \
    const int nacc = 2 + ndim * nbins;                                                                            \
    if (precision == 0) {                                                                                         \
      *smem = MeAccLayout<NG, double>::total(nacc);                                                               \
      e = cudaFuncSetAttribute(k_me_acc<NG, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem));    \
      if (e != cudaSuccess) return e;                                                                             \
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_me_acc<NG, double>, kThreads, *smem);          \
    }                                                                                                             \
    *smem = MeAccLayout<NG, float>::total(nacc);                                                                  \
    e = cudaFuncSetAttribute(k_me_acc<NG, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem));       \
    if (e != cudaSuccess) return e;                                                                               \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_me_acc<NG, float>, kThreads, *smem);             \
  }                                                                                                               \
  template <>                                                                                                     \
  cudaError_t launch_chunk<NG>(int precision, const SampleParams& sp, const MeParams& mp, const double* edges,    \
                               int64_t first_event, int64_t n, int64_t C, void* rec_base, uint64_t seed, int iter, \
                               int accumulate, double* partials, unsigned long long* counters, double* w_out,     \
                               int grid, cudaStream_t s, cudaEvent_t* ev, int me_warps) {                         \
    const int nacc = 2 + sp.ndim * sp.nbins;                                                                      \
    const size_t esm = sizeof(double) * sp.ndim * (sp.nbins + 1);                                                 \
    int dev = 0, sms = 0;                                                                                         \
    cudaGetDevice(&dev);                                                                                          \
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);                                           \
    const int64_t need = (n + kThreads - 1) / kThreads;                                                           \
    const int sgrid = int(need < int64_t(sms) * 16 ? need : int64_t(sms) * 16);                                  \
    if (precision == 0) {                                                                                         \
      RecordView<double> rec = RecordView<double>::carve(rec_base, sp.n_final, sp.ndim, C);                       \
      cudaError_t e = cudaMemsetAsync(rec.count, 0, 2 * sizeof(unsigned), s);                                    \
      if (e != cudaSuccess) return e;                                                                             \
      if (ev) cudaEventRecord(ev[0], s);                                                                          \
      k_sample_rec<double><<<sgrid, kThreads, esm, s>>>(sp, edges, first_event, n, seed, iter, rec, w_out);       \
      if (ev) cudaEventRecord(ev[1], s);                                                                          \
      k_me_acc<NG, double><<<grid, kThreads, MeAccLayout<NG, double>::total(nacc), s>>>(                          \
          mp, sp.ndim, sp.nbins, rec, accumulate, partials, counters, w_out);                                     \
      if (ev) cudaEventRecord(ev[2], s);                                                                          \
    } else {                                                                                                      \
      RecordView<float> rec = RecordView<float>::carve(rec_base, sp.n_final, sp.ndim, C);                         \
      cudaError_t e = cudaMemsetAsync(rec.count, 0, 2 * sizeof(unsigned), s);                                     \
      if (e != cudaSuccess) return e;                                                                             \
      if (ev) cudaEventRecord(ev[0], s);                                                                          \
      k_sample_rec<float><<<sgrid, kThreads, esm, s>>>(sp, edges, first_event, n, seed, iter, rec, w_out);        \
      if (ev) cudaEventRecord(ev[1], s);                                                                          \
      if (me_warps > 0) {                                                                                         \
        e = launch_me_acc_shape(me_warps, mp, sp.n_final, sp.ndim, sp.nbins, rec_base, C, accumulate, partials,  \
                                counters, w_out, grid, s);                                                        \
        if (e != cudaSuccess) return e;                                                                           \
      } else {                                                                                                    \
        k_me_acc<NG, float><<<grid, kThreads, MeAccLayout<NG, float>::total(nacc), s>>>(                          \
            mp, sp.ndim, sp.nbins, rec, accumulate, partials, counters, w_out);                                   \
      }                                                                                                           \
      if (ev) cudaEventRecord(ev[2], s);                                                                          \
    }                                                                                                             \
    return cudaGetLastError();                                                                                    \
  }                                                                                                               \
  template <>                                                                                                     \
  cudaError_t launch_me_acc<NG>(int precision, const MeParams& mp, int n_final, int ndim, int nbins,              \
                                void* rec_base, int64_t C, int accumulate, double* partials,                      \
                                unsigned long long* counters, double* w_out, int grid, cudaStream_t s) {          \
    const int nacc = 2 + ndim * nbins;                                                                            \
    if (precision == 0) {                                                                                         \
      RecordView<double> rec = RecordView<double>::carve(rec_base, n_final, ndim, C);                             \
      k_me_acc<NG, double><<<grid, kThreads, MeAccLayout<NG, double>::total(nacc), s>>>(                          \
          mp, ndim, nbins, rec, accumulate, partials, counters, w_out);                                           \
    } else {                                                                                                      \
      RecordView<float> rec = RecordView<float>::carve(rec_base, n_final, ndim, C);                               \
      k_me_acc<NG, float><<<grid, kThreads, MeAccLayout<NG, float>::total(nacc), s>>>(                            \
          mp, ndim, nbins, rec, accumulate, partials, counters, w_out);                                           \
    }                                                                                                             \
    return cudaGetLastError();                                                                                    \
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
