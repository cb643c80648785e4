// Reverse-mode derivative (adjoint) of one event's |M|^2 with respect to the
// momenta, m_t and Gamma_t (arXiv:2211.14056, Sec. 2 notes that the device
// operator has no derivative and that adding one is straightforward).
//
// One reverse sweep per event, recomputing instead of storing: the lane group
// rebuilds the mask table and the gluon sub-currents G(B), every lane walks
// its quark line to get its colour-ordered amplitudes J, the colour form gives
// Jb = 2 norm C J, and the lanes walk the quark line again, depth first,
// propagating adjoints from every amplitude back through the suffix currents
// R(S) on the current path (held in registers with their adjoints) into the
// adjoints of the sub-currents (accumulated in shared memory), of the
// propagator momenta, m_t, Gamma_t and the external spinors.  The gluon
// levels are then reversed from the longest blocks down to the polarisation
// vectors.  Derivatives of the external wavefunctions and of the propagator
// factors are taken locally (dual numbers over the few inputs of each) and
// contracted with their adjoints.
//
// Convention: for the real result f and a complex intermediate z = x + i y,
// zb = df/dx + i df/dy; then z = a w gives wb += conj(a) zb, and a real
// parameter t with dz/dt = z' gets tb += Re(conj(z') zb).
#pragma once
#include "mf_gen_adj.cuh"
#include "mf_kernels.cuh"

namespace mf {

// f(std::integral_constant<int, i>) for i = 0 .. N-1, each call inlined with
// its index a compile-time constant
template <int I, int N, typename F> __device__ __forceinline__ void static_for_from(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for_from<I + 1, N>(f);
  }
}
template <int N, typename F> __device__ __forceinline__ void static_for(F&& f) { static_for_from<0, N>(f); }

// conj(a) * b and acc + conj(a) * b
template <typename T> __device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b) {
  return {fma(a.r, b.r, a.i * b.i), fma(a.r, b.i, -(a.i * b.r))};
}
template <typename T> __device__ __forceinline__ cplx<T> cfmac(cplx<T> a, cplx<T> b, cplx<T> acc) {
  return {fma(a.r, b.r, fma(a.i, b.i, acc.r)), fma(a.r, b.i, fma(-a.i, b.r, acc.i))};
}
// Re(conj(a) b)
template <typename T> __device__ __forceinline__ T redot(cplx<T> a, cplx<T> b) { return fma(a.r, b.r, a.i * b.i); }

// o = (G-slash) R: accumulate Gb and Rb from ob
template <typename T>
__device__ __forceinline__ void adj_apply(const V4<T>& G, const S4<T>& R, const S4<T>& ob, V4<T>& Gb, S4<T>& Rb) {
  const Slash<T> s = make_slash(G);
  Rb.c[0] = cfmac(s.a, ob.c[2], cfmac(s.c, ob.c[3], Rb.c[0]));
  Rb.c[1] = cfmac(s.d, ob.c[2], cfmac(s.b, ob.c[3], Rb.c[1]));
  Rb.c[2] = cfmac(s.b, ob.c[0], cfmac(-s.c, ob.c[1], Rb.c[2]));
  Rb.c[3] = cfmac(-s.d, ob.c[0], cfmac(s.a, ob.c[1], Rb.c[3]));
  const cplx<T> ab = cfmac(R.c[3], ob.c[1], cmulc(R.c[0], ob.c[2]));
  const cplx<T> bb = cfmac(R.c[2], ob.c[0], cmulc(R.c[1], ob.c[3]));
  const cplx<T> cb = cfmac(R.c[0], ob.c[3], -cmulc(R.c[2], ob.c[1]));
  const cplx<T> db = cfmac(R.c[1], ob.c[2], -cmulc(R.c[3], ob.c[0]));
  Gb.c[0] = Gb.c[0] + ab + bb;
  Gb.c[3] = Gb.c[3] + ab - bb;
  Gb.c[1] = Gb.c[1] + cb + db;
  Gb.c[2] = Gb.c[2] + times_i(db - cb);
}

// o = f (P-slash + m) X (quark_prop_f): Xb, Pb, mb and fb from ob
template <typename T>
__device__ __forceinline__ void adj_prop(const R4<T>& P, T m, cplx<T> f, const S4<T>& X, const S4<T>& ob, S4<T>& Xb,
                                         R4<T>& Pb, T& mb, cplx<T>& fb) {
  const T a = P.v[0] + P.v[3], b = P.v[0] - P.v[3];
  const cplx<T> c = {P.v[1], P.v[2]}, d = {P.v[1], -P.v[2]};
  S4<T> y;
  y.c[0] = rfma(b, X.c[2], rfma(m, X.c[0], -(d * X.c[3])));
  y.c[1] = rfma(a, X.c[3], rfma(m, X.c[1], -(c * X.c[2])));
  y.c[2] = rfma(a, X.c[0], rfma(m, X.c[2], d * X.c[1]));
  y.c[3] = rfma(b, X.c[1], rfma(m, X.c[3], c * X.c[0]));
  cplx<T> yb[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    yb[k] = cmulc(f, ob.c[k]);
    fb = cfmac(y.c[k], ob.c[k], fb);
  }
  Xb.c[0] = rfma(m, yb[0], rfma(a, yb[2], cmulc(c, yb[3])));
  Xb.c[1] = rfma(m, yb[1], rfma(b, yb[3], cmulc(d, yb[2])));
  Xb.c[2] = rfma(b, yb[0], rfma(m, yb[2], -cmulc(c, yb[1])));
  Xb.c[3] = rfma(a, yb[1], rfma(m, yb[3], -cmulc(d, yb[0])));
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 4; ++k) s += redot(X.c[k], yb[k]);
  mb += s;
  const T ab = redot(X.c[3], yb[1]) + redot(X.c[0], yb[2]);
  const T bb = redot(X.c[2], yb[0]) + redot(X.c[1], yb[3]);
  const cplx<T> cb = cmulc(X.c[0], yb[3]) - cmulc(X.c[2], yb[1]);
  const cplx<T> db = cmulc(X.c[1], yb[2]) - cmulc(X.c[3], yb[0]);
  Pb.v[0] += ab + bb;
  Pb.v[3] += ab - bb;
  Pb.v[1] += cb.r + db.r;
  Pb.v[2] += cb.i - db.i;
}

// acc -= sg O3(GL, GR, PL, PR) (o3_sub) with accb given: GLb, GRb, PLb, PRb
template <typename T>
__device__ __forceinline__ void adj_o3(const V4<T>& GL, const V4<T>& GR, const R4<T>& PL, const R4<T>& PR, T sg,
                                       const V4<T>& accb, V4<T>& GLb, V4<T>& GRb, R4<T>& PLb, R4<T>& PRb) {
  R4<T> a, b, c;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a.v[k] = PR.v[k] - PL.v[k];
    b.v[k] = fma(T(2), PR.v[k], PL.v[k]);
    c.v[k] = fma(T(2), PL.v[k], PR.v[k]);
  }
  const cplx<T> s0 = mdot(GL, GR), s1 = mdot(b, GL), s2 = mdot(c, GR);
  cplx<T> s0b = {T(0), T(0)}, s1b = {T(0), T(0)}, s2b = {T(0), T(0)};
  R4<T> ab;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const cplx<T> ob = -sg * accb.c[k];     // adjoint of O3 component k
    s0b = rfma(a.v[k], ob, s0b);
    ab.v[k] = redot(s0, ob);
    GRb.c[k] = GRb.c[k] - cmulc(s1, ob);
    s1b = s1b - cmulc(GR.c[k], ob);
    GLb.c[k] = cfmac(s2, ob, GLb.c[k]);
    s2b = cfmac(GL.c[k], ob, s2b);
  }
  R4<T> bb, cbr;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const T g = k == 0 ? T(1) : T(-1);
    GLb.c[k] = cfmac(GR.c[k], g * s0b, GLb.c[k]);
    GRb.c[k] = cfmac(GL.c[k], g * s0b, GRb.c[k]);
    GLb.c[k] = rfma(g * b.v[k], s1b, GLb.c[k]);
    bb.v[k] = g * redot(GL.c[k], s1b);
    GRb.c[k] = rfma(g * c.v[k], s2b, GRb.c[k]);
    cbr.v[k] = g * redot(GR.c[k], s2b);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    PLb.v[k] += -ab.v[k] + bb.v[k] + T(2) * cbr.v[k];
    PRb.v[k] += ab.v[k] + T(2) * bb.v[k] + cbr.v[k];
  }
}

// acc += sg [2 (L.R) M - (L.M) R - (M.R) L] (o4_add) with accb given
template <typename T>
__device__ __forceinline__ void adj_o4(const V4<T>& GL, const V4<T>& GM, const V4<T>& GR, T sg, const V4<T>& accb,
                                       V4<T>& GLb, V4<T>& GMb, V4<T>& GRb) {
  const cplx<T> lr = mdot(GL, GR), lm = mdot(GL, GM), mr = mdot(GM, GR);
  cplx<T> lrb = {T(0), T(0)}, lmb = {T(0), T(0)}, mrb = {T(0), T(0)};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const cplx<T> ob = sg * accb.c[k];
    GMb.c[k] = cfmac(T(2) * lr, ob, GMb.c[k]);
    lrb = cfmac(T(2) * GM.c[k], ob, lrb);
    GRb.c[k] = GRb.c[k] - cmulc(lm, ob);
    lmb = lmb - cmulc(GR.c[k], ob);
    GLb.c[k] = GLb.c[k] - cmulc(mr, ob);
    mrb = mrb - cmulc(GL.c[k], ob);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const T g = k == 0 ? T(1) : T(-1);
    GLb.c[k] = cfmac(GR.c[k], g * lrb, cfmac(GM.c[k], g * lmb, GLb.c[k]));
    GRb.c[k] = cfmac(GL.c[k], g * lrb, cfmac(GM.c[k], g * mrb, GRb.c[k]));
    GMb.c[k] = cfmac(GL.c[k], g * lmb, cfmac(GR.c[k], g * mrb, GMb.c[k]));
  }
}

// amplitude planes of the adjoint kernel: [re/im][sigma * 2 + top helicity][32 lanes]
template <int NG> constexpr int kAdjPlane = TTNG<NG>::NPERM * 2 * 32;

// Per-lane accumulators of the momentum adjoints (registers; every index is
// a compile-time constant): row i*4 + c holds d|M|^2/dp[i][c] for the
// momenta in MadGraph order, then the explicit d/dm_t and d/d(m_t Gamma_t).
template <int NG> struct AdjRows {
  static constexpr int NEXT = NG + 2;
  static constexpr int MB = 4 * NEXT, MWB = 4 * NEXT + 1, N = 4 * NEXT + 2;
};
template <int NG, typename T> struct AdjAcc { T r[AdjRows<NG>::N]; };

template <int NG, typename T> __device__ __forceinline__ void acc_row(AdjAcc<NG, T>& pb, int row, T x) { pb.r[row] += x; }

// Kb for K = sum of the outgoing-convention gluon momenta q_g (g in msk),
// q_g = -p for the incoming gluons g = 0, 1 (legs 0, 1), +p for legs 4..
template <int NG, typename T> __device__ __forceinline__ void add_mask(AdjAcc<NG, T>& pb, unsigned msk, const R4<T>& Kb) {
#pragma unroll
  for (int g = 0; g < NG; ++g)
    if ((msk >> g) & 1u) {
      const int leg = g < 2 ? g : g + 2;
      const T s = g < 2 ? T(-1) : T(1);
#pragma unroll
      for (int c = 0; c < 4; ++c) acc_row<NG, T>(pb, leg * 4 + c, s * Kb.v[c]);
    }
}

// adjoint of the propagator factor f = -1/(den + i m Gamma), den = P^2 - m^2
// with P = q_tbar + K(msk) (= -Ptab[msk]); a Ptab adjoint Ptb is folded in
template <int NG, typename T>
__device__ __forceinline__ void chain_prop(AdjAcc<NG, T>& pb, unsigned msk, const R4<T>& Ptab, cplx<T> f, cplx<T> fb,
                                           const R4<T>& Ptb, T m) {
  const cplx<T> f2 = f * f;                  // d f / d z = 1 / z^2 = f^2
  const cplx<T> zb = cmulc(f2, fb);
  const T denb = zb.r, mwb = zb.i;
  R4<T> Pb;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const T g = c == 0 ? T(1) : T(-1);
    Pb.v[c] = T(2) * g * (-Ptab.v[c]) * denb - Ptb.v[c];
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) acc_row<NG, T>(pb, 3 * 4 + c, Pb.v[c]);   // q_tbar = p[3]
  add_mask<NG, T>(pb, msk, Pb);
  acc_row<NG, T>(pb, AdjRows<NG>::MB, T(-2) * m * denb);
  acc_row<NG, T>(pb, AdjRows<NG>::MWB, mwb);
}

// d(spinor)/d(E, px, py, pz, m) contracted with the spinor's adjoint
template <int NG, typename T, typename F>
__device__ __forceinline__ void chain_spinor(AdjAcc<NG, T>& pb, int leg, const T (&p)[4], T m, const S4<T>& sb, F&& fn) {
  using D = Dual<T, 5>;
  R4<D> pd;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    pd.v[c] = D(p[c]);
    pd.v[c].d[c] = T(1);
  }
  D md = D(m);
  md.d[4] = T(1);
  const S4<D> s = fn(pd, md);
  T g[5] = {T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 5; ++j) g[j] += s.c[k].r.d[j] * sb.c[k].r + s.c[k].i.d[j] * sb.c[k].i;
#pragma unroll
  for (int c = 0; c < 4; ++c) acc_row<NG, T>(pb, leg * 4 + c, g[c]);
  acc_row<NG, T>(pb, AdjRows<NG>::MB, g[4]);
}

// Reverse depth-first walk (see quark_walk for the forward recursion).  The
// forward pass (ADJ = false) stores the amplitudes J; the reverse pass
// (ADJ = true) reads Jb in their place, recomputes every R(S) on the way down
// and, after a node's subtree, propagates the node's adjoint Rb[LV] into the
// sub-currents (atomically into Gb), the propagator inputs and Rb of its
// ancestors.
template <typename T> struct AdjCtx {
  const cplx<T>* Gs;
  cplx<T>* Gb;
  const R4<T>* Ptab;
  const cplx<T>* qf;
  uint64_t pk;
  S4<T> ub0, ub1, ubb0, ubb1;
  T m;
  T* J;          // this lane's column of the J (or Jb) planes
  unsigned gl;   // lane within the event's group
};

// The sub-current adjoints Gb are stored component-major like Gs, but with a
// component stride of one entry more than they hold: where the entry count is
// a multiple of 16 complex numbers (128 or 320 for four gluons) the four
// components of one entry would share a bank, and the lanes that add
// different components of one entry at once would conflict.
//
// With four gluons the adjoints of the four-gluon blocks (192 of the 320
// entries) are not in Gb: each such block is used only by the completions of
// its two colour orderings, and its adjoint is kept in the amplitude rows of
// the ordering the walk completes first (rows that are dead once that
// completion has read its Jb); see g4_leaf_add.  The shared footprint of a
// warp drops from 33.5 to 26.7 KB, which lets eight one-warp CTAs share an SM
// instead of six.
template <int NG> constexpr bool kG4InJ = NG == 4;
template <int NG>
constexpr int kGbEntries = kG4InJ<NG> ? TTNG<NG>::NSTORE - ((TTNG<NG>::FIRST[NG + 1] - TTNG<NG>::FIRST[NG]) << NG)
                                      : TTNG<NG>::NSTORE;
template <int NG> constexpr int kGbStride = kGbEntries<NG> + 1;

template <int NG, typename T>
__device__ __forceinline__ V4<T> gb_load(const cplx<T>* Gb, int pos) {
  V4<T> g;
#pragma unroll
  for (int k = 0; k < 4; ++k) g.c[k] = Gb[k * kGbStride<NG> + pos];
  return g;
}

// Add a lane's adjoint of a sub-current it used.  The stored position depends
// only on the helicities of the block's own gluons, so the lanes that differ
// in the other gluons' or the antitop's helicity (the R = popcount(other) bits
// of `other`) add to the same entry.  Their sum is formed by a reduce-scatter
// over those lane bits: over each of the first min(R, 3) bits a lane keeps
// half of its remaining components and exchanges the other half (4 + 2 + 1
// shuffles instead of 8 per bit), over any further bit it exchanges its last
// component; then every lane whose further bits are zero holds the complete
// sums of 8 >> min(R, 3) components and adds them (the entry's eight
// additions spread over 2^min(R, 3) lanes).
template <int S, typename T>
__device__ __forceinline__ void gb_split(T (&v)[8], unsigned b, unsigned gl, int& coff) {
  const bool up = (gl >> b) & 1u;
#pragma unroll
  for (int i = 0; i < S / 2; ++i) {
    const T send = up ? v[i] : v[i + S / 2];
    const T keep = up ? v[i + S / 2] : v[i];
    v[i] = keep + shfl_xor_any(0xffffffffu, send, 1 << b);
  }
  if (up) coff += S / 2;
}

template <int NG, int R, typename T>
__device__ __forceinline__ void gb_scatter_add(T (&v)[8], unsigned other, unsigned gl, cplx<T>* Gb, int pos, T sg,
                                               bool act = true) {
  constexpr int M = R < 3 ? R : 3;
  constexpr int S = 8 >> M;
  unsigned rem = other;
  int coff = 0;
  if constexpr (M >= 1) { gb_split<8, T>(v, unsigned(__ffs(rem) - 1), gl, coff); rem &= rem - 1u; }
  if constexpr (M >= 2) { gb_split<4, T>(v, unsigned(__ffs(rem) - 1), gl, coff); rem &= rem - 1u; }
  if constexpr (M >= 3) { gb_split<2, T>(v, unsigned(__ffs(rem) - 1), gl, coff); rem &= rem - 1u; }
  const unsigned extra = rem;
#pragma unroll
  for (int e = 0; e < R - M; ++e) {
    const unsigned b = unsigned(__ffs(rem) - 1);
    rem &= rem - 1u;
#pragma unroll
    for (int i = 0; i < S; ++i) v[i] += shfl_xor_any(0xffffffffu, v[i], 1 << b);
  }
  if (!act || (gl & extra) != 0u) return;
  T* base = reinterpret_cast<T*>(Gb);
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const int c = coff + i;   // component c: k = c / 2, real (c even) or imaginary part
    atomicAdd(base + 2 * ((c >> 1) * kGbStride<NG> + pos) + (c & 1), sg * v[i]);
  }
}

// BL = the block's gluon count, a compile-time constant at every call site:
// the walk's m-th block of a path (m = 0, 1, ...) holds m + 1 gluons (the
// path tables are built that way), so each site inlines one reduction form.
template <int NG, int BL, typename T>
__device__ __forceinline__ void gb_add(const AdjCtx<T>& cx, uint16_t ref, V4<T> g) {
  static_assert(BL >= 1 && BL <= NG, "a block holds 1 .. NG gluons");
  const unsigned mb = ref_mask(ref);
  const unsigned other = ((2u << NG) - 1u) & ~mb;   // NG + 1 - BL lane bits
  const unsigned idx = unsigned(cx.pk >> (4 * mb)) & 15u;
  const int pos = ref_off(ref) + int(idx);
  const T sg = ref_neg(ref) ? T(-1) : T(1);
  T v[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = g.c[k].r;
    v[2 * k + 1] = g.c[k].i;
  }
  gb_scatter_add<NG, NG + 1 - BL, T>(v, other, cx.gl, cx.Gb, pos, sg);
}

// Position, in the warp's amplitude planes, of value c (component c / 2, real
// or imaginary part by c & 1) of helicity entry idx of a four-gluon block
// kept in the rows of colour ordering `slot`: the rows (slot, top helicity
// 0/1) of both planes, 32 words each, in half rows of 16 entries; half
// (c / 4) ^ parity of the block, so that the two antitop lanes' stores of
// one entry, and the two blocks of a round of the reversed gluon level,
// fall in different banks.
__device__ __forceinline__ int g4_off(int slot, int c, unsigned par, unsigned idx) {
  const int row = c & 3, half = (c >> 2) ^ int(par);
  return (row >> 1) * kAdjPlane<4> + (slot * 2 + (row & 1)) * 32 + half * 16 + int(idx);
}

// A completion's adjoint of its four-gluon block: summed over the antitop
// lane bit (each lane keeps four of the eight values), then stored, at the
// block's first completion, or added, at its second, by the lane that owns
// each value (the same lane both times, so no atomics).  The first
// completion writes over the rows it has just read, hence the warp barrier.
template <typename T>
__device__ __forceinline__ void g4_leaf_add(const AdjCtx<T>& cx, int path, uint16_t ref, const V4<T>& g) {
  const unsigned e = kG4Leaf4[path];
  const int slot = int(e & 31u);
  const unsigned par = (e >> 5) & 1u;
  const T sg = ref_neg(ref) ? T(-1) : T(1);
  const unsigned idx = unsigned(cx.pk >> (4 * ref_mask(ref))) & 15u;
  T v[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = g.c[k].r;
    v[2 * k + 1] = g.c[k].i;
  }
  int coff = 0;
  gb_split<8, T>(v, 4u, cx.gl, coff);
  T* base = cx.J - (threadIdx.x & 31);
  __syncwarp();
  if (e & 0x80u) {
#pragma unroll
    for (int i = 0; i < 4; ++i) base[g4_off(slot, coff + i, par, idx)] = sg * v[i];
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) base[g4_off(slot, coff + i, par, idx)] += sg * v[i];
  }
}

template <int NG, typename T>
__device__ __forceinline__ V4<T> adj_block(const AdjCtx<T>& cx, uint16_t ref) {
  const unsigned idx = unsigned(cx.pk >> (4 * ref_mask(ref))) & 15u;
  V4<T> g = gs_load<NG, T>(cx.Gs, ref_off(ref) + int(idx));
  if (ref_neg(ref)) g = neg(g);
  return g;
}

template <int NG, int LV, bool ADJ, typename T>
__device__ __forceinline__ void adj_walk(int parent, S4<T> (&R)[NG], S4<T> (&Rb)[NG], AdjCtx<T>& cx,
                                         AdjAcc<NG, T>& pb) {
  using PT = Paths<NG>;
  const int first = PT::template first<LV>(parent);
#pragma unroll 1
  for (int k = 0; k <= NG - LV; ++k) {
    const int path = first + k;
    const uint8_t msk = PT::template mask<LV>(path);
    S4<T> Xd = apply(make_slash(adj_block<NG, T>(cx, PT::template blk<LV>(path, 0))), R[LV - 1]);
#pragma unroll
    for (int m = 1; m < LV; ++m)
      apply_acc(make_slash(adj_block<NG, T>(cx, PT::template blk<LV>(path, m))), R[LV - 1 - m], Xd);
    R[LV] = quark_prop_f(cx.Ptab[msk], cx.m, cx.qf[msk], Xd);
    if constexpr (ADJ) {
#pragma unroll
      for (int c = 0; c < 4; ++c) Rb[LV].c[c] = {T(0), T(0)};
    }
    if constexpr (LV < NG - 1) {
      adj_walk<NG, LV + 1, ADJ, T>(path, R, Rb, cx, pb);
    } else {
      {
        S4<T> W = apply(make_slash(adj_block<NG, T>(cx, PT::final_blk(path, 0))), R[NG - 1]);
#pragma unroll
        for (int m = 1; m < NG; ++m)
          apply_acc(make_slash(adj_block<NG, T>(cx, PT::final_blk(path, m))), R[NG - 1 - m], W);
        const int sig = PT::final_sigma(path);
        T* j = cx.J + (sig * 2) * 32;
        if constexpr (!ADJ) {
          const cplx<T> j0 = rowdot(cx.ub0, W), j1 = rowdot(cx.ub1, W);
          j[0] = j0.r;
          j[kAdjPlane<NG>] = j0.i;
          j[32] = j1.r;
          j[32 + kAdjPlane<NG>] = j1.i;
        } else {
          const cplx<T> jb0 = {j[0], j[kAdjPlane<NG>]}, jb1 = {j[32], j[32 + kAdjPlane<NG>]};
          S4<T> Wb;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            Wb.c[c] = cfmac(cx.ub1.c[c], jb1, cmulc(cx.ub0.c[c], jb0));
            cx.ubb0.c[c] = cfmac(W.c[c], jb0, cx.ubb0.c[c]);
            cx.ubb1.c[c] = cfmac(W.c[c], jb1, cx.ubb1.c[c]);
          }
          static_for<NG>([&](auto mc) {
            constexpr int m = decltype(mc)::value;
            const uint16_t ref = PT::final_blk(path, m);
            V4<T> gb;
#pragma unroll
            for (int c = 0; c < 4; ++c) gb.c[c] = {T(0), T(0)};
            adj_apply(adj_block<NG, T>(cx, ref), R[NG - 1 - m], Wb, gb, Rb[NG - 1 - m]);
            if constexpr (m == NG - 1 && kG4InJ<NG>)
              g4_leaf_add<T>(cx, path, ref, gb);
            else
              gb_add<NG, m + 1, T>(cx, ref, gb);
          });
        }
      }
    }
    if constexpr (ADJ) {
      // node adjoint: R[LV] = f (P-slash + m) X, X = sum_m G_m-slash R[LV-1-m];
      // in FP32 the node above the completions keeps its X over its one
      // completion; the higher nodes and FP64 recompute it (more live values:
      // spills)
      S4<T> X;
      if constexpr (LV == NG - 1 && std::is_same<T, float>::value) {
        X = Xd;
      } else {
        X = apply(make_slash(adj_block<NG, T>(cx, PT::template blk<LV>(path, 0))), R[LV - 1]);
#pragma unroll
        for (int m = 1; m < LV; ++m)
          apply_acc(make_slash(adj_block<NG, T>(cx, PT::template blk<LV>(path, m))), R[LV - 1 - m], X);
      }
      S4<T> Xb;
      R4<T> Ptb = {{T(0), T(0), T(0), T(0)}};
      T mb = T(0);
      cplx<T> fb = {T(0), T(0)};
      const R4<T> Pt = cx.Ptab[msk];
      const cplx<T> f = cx.qf[msk];
      adj_prop(Pt, cx.m, f, X, Rb[LV], Xb, Ptb, mb, fb);
      acc_row<NG, T>(pb, AdjRows<NG>::MB, mb);
      chain_prop<NG, T>(pb, msk, Pt, f, fb, Ptb, cx.m);
      static_for<LV>([&](auto mc) {
        constexpr int m = decltype(mc)::value;
        const uint16_t ref = PT::template blk<LV>(path, m);
        V4<T> gb;
#pragma unroll
        for (int c = 0; c < 4; ++c) gb.c[c] = {T(0), T(0)};
        adj_apply(adj_block<NG, T>(cx, ref), R[LV - 1 - m], Xb, gb, Rb[LV - 1 - m]);
        gb_add<NG, m + 1, T>(cx, ref, gb);
      });
    }
  }
}


// The forward pass (amplitudes J only) for four gluons as the |M|^2 kernel
// computes it: the two-gluon suffix currents once per event by the group
// (shared_suffixes, into R2), the three-gluon currents shared by the lane
// pairs that differ in the missing gluon's helicity (as quark_walk_paired4),
// both completions of a pair in one loop body.  J in the adjoint's layout.
template <typename T>
__device__ __forceinline__ void adj_forward_paired4(const S4<T>& v, const AdjCtx<T>& cx, const cplx<T>* R2,
                                                    unsigned H, unsigned ltb) {
  using PT = Paths<4>;
  constexpr int NR2 = WarpMem<4, T>::NR2;
  auto load_r2 = [&](int p2) {
    const uint8_t m2 = PT::template mask<2>(p2);
    const int idx = p2 * 8 + int((unsigned(cx.pk >> (4 * m2)) & 15u) | (ltb << 2));
    S4<T> r;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.c[k] = R2[k * NR2 + idx];
    return r;
  };
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
    S4<T> R[4];
    R[0] = v;
    const uint8_t m1 = PT::template mask<1>(c);
    R[1] = quark_prop_f(cx.Ptab[m1], cx.m, cx.qf[m1],
                        apply(make_slash(adj_block<4, T>(cx, PT::template blk<1>(c, 0))), v));
#pragma unroll 1
    for (int gi = 0; gi < 3; ++gi) {
      const int g = kL3Miss4[c * 3 + gi];
      const unsigned bit = (H >> g) & 1u;
      const int mine = kL3Pair4[(c * 3 + gi) * 2 + bit], other = kL3Pair4[(c * 3 + gi) * 2 + (bit ^ 1u)];
      R[2] = load_r2(mine >> 1);
      S4<T> X = apply(make_slash(adj_block<4, T>(cx, PT::template blk<3>(mine, 0))), R[2]);
      apply_acc(make_slash(adj_block<4, T>(cx, PT::template blk<3>(mine, 1))), R[1], X);
      apply_acc(make_slash(adj_block<4, T>(cx, PT::template blk<3>(mine, 2))), v, X);
      const uint8_t m3 = PT::template mask<3>(mine);
      R[3] = quark_prop_f(cx.Ptab[m3], cx.m, cx.qf[m3], X);
      S4<T> Ro;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        Ro.c[k].r = shfl_xor_any(0xffffffffu, R[3].c[k].r, 1 << g);
        Ro.c[k].i = shfl_xor_any(0xffffffffu, R[3].c[k].i, 1 << g);
      }
      int path = mine;
#pragma unroll 1
      for (int w = 0; w < 2; ++w) {
        S4<T> W = apply(make_slash(adj_block<4, T>(cx, PT::final_blk(path, 0))), R[3]);
#pragma unroll
        for (int m = 1; m < 4; ++m)
          apply_acc(make_slash(adj_block<4, T>(cx, PT::final_blk(path, m))), R[3 - m], W);
        const int sig = PT::final_sigma(path);
        T* j = cx.J + (sig * 2) * 32;
        const cplx<T> j0 = rowdot(cx.ub0, W), j1 = rowdot(cx.ub1, W);
        j[0] = j0.r;
        j[kAdjPlane<4>] = j0.i;
        j[32] = j1.r;
        j[32 + kAdjPlane<4>] = j1.i;
        if (w == 0) {
          R[2] = load_r2(other >> 1);
          R[3] = Ro;
          path = other;
        }
      }
    }
  }
}

// Add an item's adjoint of one of its sub-blocks (R = the number of the
// block's gluons outside the sub-block, a compile-time constant at every
// split).  The items of a round sit on consecutive lanes with the helicity
// index c in the low K lane bits; the items of one block whose helicities
// differ only in gluons outside the sub-block (lane bits `red`) hit the same
// entry, so they are summed by the reduce-scatter of gb_scatter_add and the
// sums added by 2^min(R, 3) of them.  Inactive lanes (past the last item;
// whole blocks of them) carry zeros through the shuffles and add nothing.
// Every lane of the group calls this.
template <int NG, int R, typename T>
__device__ __forceinline__ void gb_item_add(cplx<T>* Gb, int pos, const V4<T>& g, unsigned red, unsigned gl, bool act) {
  T v[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = g.c[k].r;
    v[2 * k + 1] = g.c[k].i;
  }
  gb_scatter_add<NG, R, T>(v, red, gl, Gb, pos, T(1), act);
}

// The s-th four-vertex split of a K-gluon block t: blocks t[:a], t[a:b],
// t[b:] in generator order (a < b); which = 0 gives a, 1 gives b.
template <int K> constexpr int o4_cut(int s, int which) {
  int i = 0;
  for (int a = 1; a < K - 1; ++a)
    for (int b = a + 1; b < K; ++b) {
      if (i == s) return which == 0 ? a : b;
      ++i;
    }
  return 0;
}

// Reverse of gluon_level<NG, K>: every item's adjoint Gb is complete (all its
// users, longer blocks and quark lines, are done); propagate it into the
// sub-blocks' adjoints, the momentum sums and 1/K^2.  Rounds of L items run
// on all lanes (idle lanes carry zero adjoints through the shuffles).
template <int NG, int K, typename T>
__device__ __forceinline__ void adj_gluon_level(const MaskTab<NG, T>& mt, const cplx<T>* Gs, cplx<T>* Gb, const T* Jw,
                                                int gl, AdjAcc<NG, T>& pb) {
  constexpr int L = Lanes<NG>::L;
  constexpr int nblk = TTNG<NG>::FIRST[K + 1] - TTNG<NG>::FIRST[K];
  constexpr int items = nblk << K;
  constexpr int n3 = K - 1;
  constexpr int n4 = (K - 1) * (K - 2) / 2;
#pragma unroll 1
  for (int base = 0; base < items; base += L) {
    const int it = base + gl;
    const bool act = it < items;
    const int bl = act ? it >> K : 0;
    const unsigned c = unsigned(it) & ((1u << K) - 1u);
    const int b = TTNG<NG>::FIRST[K] + bl;
    const unsigned mb = blk_mask<NG>()[b];
    const unsigned H = pdep_mask<NG>(c, mb);
    const int pos = blk_off<NG>()[b] + int(c);
    const V4<T> G = gs_load<NG, T>(Gs, pos);
    V4<T> Gbar;
    if constexpr (K == NG && kG4InJ<NG>) {
      // kept in the amplitude rows (g4_leaf_add)
      const int slot = kG4Slot4[bl];
      const unsigned par = unsigned(bl) & 1u;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        Gbar.c[k] = {Jw[g4_off(slot, 2 * k, par, c)], Jw[g4_off(slot, 2 * k + 1, par, c)]};
    } else {
      Gbar = gb_load<NG, T>(Gb, pos);
    }
    if (!act) {
#pragma unroll
      for (int k = 0; k < 4; ++k) Gbar.c[k] = {T(0), T(0)};
    }
    const T ginv = mt.ginv[mb];
    // G = ginv acc: d/d(ginv) = Re(conj(acc) Gb) = Re(conj(G) Gb) / ginv, ginv = 1/K^2
    T gib = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) gib += redot(G.c[k], Gbar.c[k]);
    const T k2b = -ginv * gib;
    const R4<T> Kv = mt.qsum[mb];
    R4<T> Kb;
#pragma unroll
    for (int k = 0; k < 4; ++k) Kb.v[k] = T(2) * (k == 0 ? T(1) : T(-1)) * Kv.v[k] * k2b;
    add_mask<NG, T>(pb, mb, Kb);
    V4<T> accb;
#pragma unroll
    for (int k = 0; k < 4; ++k) accb.c[k] = ginv * Gbar.c[k];
    // one inlined body per split: each sub-block's length, hence the number of
    // lane bits its adjoint is summed over, is a compile-time constant
    const uint16_t* t3 = o3_table<NG, K>() + bl * n3 * 2;
    static_for<n3>([&](auto sc) {
      constexpr int sp = decltype(sc)::value;   // blocks t[:sp+1], t[sp+1:]
      const uint16_t rl = t3[2 * sp], rr = t3[2 * sp + 1];
      const V4<T> GL = load_block<NG, T>(Gs, rl, H), GR = load_block<NG, T>(Gs, rr, H);
      const R4<T> PL = mt.qsum[ref_mask(rl)], PR = mt.qsum[ref_mask(rr)];
      V4<T> GLb, GRb;
#pragma unroll
      for (int k = 0; k < 4; ++k) GLb.c[k] = GRb.c[k] = {T(0), T(0)};
      R4<T> PLb = {{T(0), T(0), T(0), T(0)}}, PRb = {{T(0), T(0), T(0), T(0)}};
      adj_o3(GL, GR, PL, PR, (ref_neg(rl) != ref_neg(rr)) ? T(-1) : T(1), accb, GLb, GRb, PLb, PRb);
      gb_item_add<NG, K - sp - 1, T>(Gb, ref_off(rl) + int(pext_mask<NG>(H, ref_mask(rl))), GLb,
                                     pext_mask<NG>(mb & ~ref_mask(rl), mb), unsigned(gl), act);
      gb_item_add<NG, sp + 1, T>(Gb, ref_off(rr) + int(pext_mask<NG>(H, ref_mask(rr))), GRb,
                                 pext_mask<NG>(mb & ~ref_mask(rr), mb), unsigned(gl), act);
      add_mask<NG, T>(pb, ref_mask(rl), PLb);
      add_mask<NG, T>(pb, ref_mask(rr), PRb);
    });
    if constexpr (K >= 3) {
      const uint16_t* t4 = o4_table<NG, K>() + bl * n4 * 3;
      static_for<n4>([&](auto sc) {
        constexpr int sp = decltype(sc)::value;
        constexpr int a = o4_cut<K>(sp, 0), b = o4_cut<K>(sp, 1);   // blocks t[:a], t[a:b], t[b:]
        const uint16_t r0 = t4[3 * sp], r1 = t4[3 * sp + 1], r2 = t4[3 * sp + 2];
        const V4<T> GL = load_block<NG, T>(Gs, r0, H), GM = load_block<NG, T>(Gs, r1, H),
                    GR = load_block<NG, T>(Gs, r2, H);
        V4<T> GLb, GMb, GRb;
#pragma unroll
        for (int k = 0; k < 4; ++k) GLb.c[k] = GMb.c[k] = GRb.c[k] = {T(0), T(0)};
        adj_o4(GL, GM, GR, (ref_neg(r0) ^ ref_neg(r1) ^ ref_neg(r2)) ? T(-1) : T(1), accb, GLb, GMb, GRb);
        gb_item_add<NG, K - a, T>(Gb, ref_off(r0) + int(pext_mask<NG>(H, ref_mask(r0))), GLb,
                                  pext_mask<NG>(mb & ~ref_mask(r0), mb), unsigned(gl), act);
        gb_item_add<NG, K - (b - a), T>(Gb, ref_off(r1) + int(pext_mask<NG>(H, ref_mask(r1))), GMb,
                                        pext_mask<NG>(mb & ~ref_mask(r1), mb), unsigned(gl), act);
        gb_item_add<NG, b, T>(Gb, ref_off(r2) + int(pext_mask<NG>(H, ref_mask(r2))), GRb,
                              pext_mask<NG>(mb & ~ref_mask(r2), mb), unsigned(gl), act);
      });
    }
  }
}

// Shared memory of one warp of the adjoint kernel: per event of the warp the
// sub-currents, their adjoints and the mask table; per lane the amplitude
// planes (J, then Jb).
template <int NG, typename T> struct AdjMem {
  static constexpr int EPW = Lanes<NG>::EPW;
  static constexpr size_t gs_bytes = sizeof(cplx<T>) * 4 * TTNG<NG>::NSTORE * EPW;
  static constexpr size_t gb_bytes = sizeof(cplx<T>) * 4 * kGbStride<NG> * EPW;
  static constexpr size_t gb_off = gs_bytes;
  static constexpr size_t pt_off = gb_off + gb_bytes;
  static constexpr size_t j_off = (pt_off + MaskTab<NG, T>::bytes * EPW + 15) & ~size_t(15);
  static constexpr size_t bytes = (j_off + sizeof(T) * 2 * kAdjPlane<NG> + 15) & ~size_t(15);
};

// |M|^2 of the group's event (every lane returns it) and, on return, the
// group-summed adjoint rows d|M|^2/dp[i][c], d/dm_t, d/d(m_t Gamma_t) in out[]
// (all lanes).  norm includes 1/D of the colour matrix C = num / D.
template <int NG, typename T>
__device__ __forceinline__ T adj_group_me2(const T (&p)[NG + 2][4], unsigned char* wm, int group, int gl, T mt, T mw,
                                           T norm, T (&out)[AdjRows<NG>::N]) {
  using AM = AdjMem<NG, T>;
  constexpr int L = Lanes<NG>::L, NP = TTNG<NG>::NPERM, NS = TTNG<NG>::NSTORE, NR = AdjRows<NG>::N;
  const int lane = threadIdx.x & 31;
  cplx<T>* Gs = reinterpret_cast<cplx<T>*>(wm) + group * 4 * NS;
  cplx<T>* Gb = reinterpret_cast<cplx<T>*>(wm + AM::gb_off) + group * 4 * kGbStride<NG>;
  const MaskTab<NG, T> mtab(wm + AM::pt_off + group * MaskTab<NG, T>::bytes);
  T* Jw = reinterpret_cast<T*>(wm + AM::j_off) + lane;
  // four gluons: the sub-current adjoint store holds the two-gluon suffix
  // currents during the forward pass and is cleared after it
  constexpr bool kFwdPaired = NG == 4 && kShareSuffixes<T>;
  static_assert(!kFwdPaired || WarpMem<NG, T>::NR2 <= kGbStride<NG>, "R2 fits the adjoint store");
  if constexpr (!kFwdPaired)
    for (int i = gl; i < 4 * kGbStride<NG>; i += L) Gb[i] = {T(0), T(0)};
  AdjAcc<NG, T> pb;
#pragma unroll
  for (int r = 0; r < NR; ++r) pb.r[r] = T(0);
  R4<T> qtb;
#pragma unroll
  for (int c = 0; c < 4; ++c) qtb.v[c] = p[3][c];
  event_tables<NG, T>(p, mtab, Gs, gl, mt, mw);
  __syncwarp();
  gluon_level<NG, 2, T>(mtab, Gs, gl);
  if constexpr (NG >= 3) { __syncwarp(); gluon_level<NG, 3, T>(mtab, Gs, gl); }
  if constexpr (NG >= 4) { __syncwarp(); gluon_level<NG, 4, T>(mtab, Gs, gl); }
  __syncwarp();
  // this lane's quark line: amplitudes J
  const unsigned H = unsigned(gl) & ((1u << NG) - 1u);
  const int ltb = ((gl >> NG) & 1) ? 1 : -1;
  AdjCtx<T> cx;
  cx.Gs = Gs;
  cx.Gb = Gb;
  cx.Ptab = mtab.ptab;
  cx.qf = mtab.qf;
  cx.pk = 0;
#pragma unroll
  for (unsigned msk = 1; msk < (1u << NG); ++msk) cx.pk |= uint64_t(pext_mask<NG>(H, msk)) << (4 * msk);
  R4<T> pt;
#pragma unroll
  for (int c = 0; c < 4; ++c) pt.v[c] = p[2][c];
  cx.ub0 = ubar_out(pt, mt, -1);
  cx.ub1 = ubar_out(pt, mt, 1);
#pragma unroll
  for (int c = 0; c < 4; ++c) cx.ubb0.c[c] = cx.ubb1.c[c] = {T(0), T(0)};
  cx.m = mt;
  cx.J = Jw;
  cx.gl = unsigned(gl);
  S4<T> R[NG], Rb[NG];
  R[0] = v_out(qtb, mt, ltb);
  if constexpr (kFwdPaired) {
    shared_suffixes<NG, T>(Gs, mtab, qtb, mt, Gb, gl);
    __syncwarp();
    adj_forward_paired4<T>(R[0], cx, Gb, H, unsigned((gl >> NG) & 1));
    __syncwarp();   // every lane has read the suffix currents
    for (int i = gl; i < 4 * kGbStride<NG>; i += L) Gb[i] = {T(0), T(0)};
  } else {
    adj_walk<NG, 1, false, T>(0, R, Rb, cx, pb);
  }
  // colour form and its adjoint Jb = 2 norm C J (in place), per top helicity
  const int* num = colour_num_dev<NG>();
  const T js = T(2) * norm;     // norm carries the colour matrix's 1/D
  T me = T(0);
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    cplx<T> Y[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) Y[a] = {T(0), T(0)};
#pragma unroll 1
    for (int b = 0; b < NP; ++b) {
      const cplx<T> jb = {Jw[(b * 2 + h) * 32], Jw[(b * 2 + h) * 32 + kAdjPlane<NG>]};
#pragma unroll
      for (int a = 0; a < NP; ++a) Y[a] = rfma(T(num[a * NP + b]), jb, Y[a]);
    }
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      T* j = Jw + (a * 2 + h) * 32;
      me += redot(cplx<T>{j[0], j[kAdjPlane<NG>]}, Y[a]);
      j[0] = js * Y[a].r;
      j[kAdjPlane<NG>] = js * Y[a].i;
    }
  }
  me *= T(0.5) * js;
  // reverse walk, then the external spinors
#pragma unroll
  for (int c = 0; c < 4; ++c) Rb[0].c[c] = {T(0), T(0)};
  adj_walk<NG, 1, true, T>(0, R, Rb, cx, pb);
  chain_spinor<NG, T>(pb, 3, p[3], mt, Rb[0], [&](const R4<Dual<T, 5>>& q, Dual<T, 5> m) { return v_out(q, m, ltb); });
  chain_spinor<NG, T>(pb, 2, p[2], mt, cx.ubb0, [&](const R4<Dual<T, 5>>& q, Dual<T, 5> m) { return ubar_out(q, m, -1); });
  chain_spinor<NG, T>(pb, 2, p[2], mt, cx.ubb1, [&](const R4<Dual<T, 5>>& q, Dual<T, 5> m) { return ubar_out(q, m, 1); });
  __syncwarp();
  // gluon levels in reverse
  if constexpr (NG >= 4) { adj_gluon_level<NG, 4, T>(mtab, Gs, Gb, Jw - lane, gl, pb); __syncwarp(); }
  if constexpr (NG >= 3) { adj_gluon_level<NG, 3, T>(mtab, Gs, Gb, Jw - lane, gl, pb); __syncwarp(); }
  adj_gluon_level<NG, 2, T>(mtab, Gs, Gb, Jw - lane, gl, pb);
  __syncwarp();
  // polarisation vectors of the outgoing gluons (the incoming ones lie on the
  // beam axis, where eps does not depend on the momentum)
#pragma unroll
  for (int g = 2; g < NG; ++g) {
#pragma unroll
    for (int bit = 0; bit < 2; ++bit) {
      if (gl != (2 * g + bit) % L) continue;
      const V4<T> eb = gb_load<NG, T>(Gb, 2 * g + bit);
      using D = Dual<T, 3>;
      R4<D> kd;
      kd.v[0] = D(p[g + 2][0]);
#pragma unroll
      for (int c = 1; c < 4; ++c) {
        kd.v[c] = D(p[g + 2][c]);
        kd.v[c].d[c - 1] = T(1);
      }
      const V4<D> e = polarisation(kd, bit ? 1 : -1, true);
#pragma unroll
      for (int c = 1; c < 4; ++c) {
        T s = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) s += e.c[k].r.d[c - 1] * eb.c[k].r + e.c[k].i.d[c - 1] * eb.c[k].i;
        acc_row<NG, T>(pb, (g + 2) * 4 + c, s);
      }
    }
  }
  __syncwarp();
  // sum the group's lanes
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    T x = pb.r[r];
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1) x += shfl_xor_any(0xffffffffu, x, off);
    out[r] = x;
  }
#pragma unroll
  for (int off = L / 2; off > 0; off >>= 1) me += shfl_xor_any(0xffffffffu, me, off);
  __syncwarp();
  return me;
}

}  // namespace mf
