// Device-side building blocks of the tree-level helicity amplitudes:
// complex numbers, four-vectors, Dirac spinors in the chiral representation,
// external wavefunctions, vertices and propagators (arXiv:2211.14056, Sec. 2:
// "vertices, spinors or propagators" are the pieces the device operator needs).
//
// Conventions (HELAS-style, Murayama-Watanabe-Hagiwara KEK-91-11):
//   gamma^0 = [[0,1],[1,0]], gamma^k = [[0,sigma^k],[-sigma^k,0]], psi = (psi_L, psi_R);
//   metric (+,-,-,-); vectors are stored contravariant;
//   helicity label l = -1 / +1 selected by a bit (0 / 1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mf {

template <typename T> struct cplx { T r, i; };

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T r, T i) { return {r, i}; }
template <typename T> __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.r + b.r, a.i + b.i}; }
template <typename T> __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.r - b.r, a.i - b.i}; }
template <typename T> __device__ __forceinline__ cplx<T> operator-(cplx<T> a) { return {-a.r, -a.i}; }
template <typename T> __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
  return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
template <typename T> __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return {s * a.r, s * a.i}; }
// a + b*c (complex fused multiply-add, four real FMAs)
template <typename T> __device__ __forceinline__ cplx<T> cfma(cplx<T> b, cplx<T> c, cplx<T> a) {
  return {fma(b.r, c.r, fma(-b.i, c.i, a.r)), fma(b.r, c.i, fma(b.i, c.r, a.i))};
}
// a + s*b, s real
template <typename T> __device__ __forceinline__ cplx<T> rfma(T s, cplx<T> b, cplx<T> a) {
  return {fma(s, b.r, a.r), fma(s, b.i, a.i)};
}
template <typename T> __device__ __forceinline__ cplx<T> conj(cplx<T> a) { return {a.r, -a.i}; }
// i * a
template <typename T> __device__ __forceinline__ cplx<T> times_i(cplx<T> a) { return {-a.i, a.r}; }

template <typename T> struct R4 { T v[4]; };            // real four-vector (E, px, py, pz)
template <typename T> struct V4 { cplx<T> c[4]; };      // complex four-vector (contravariant)
template <typename T> struct S4 { cplx<T> c[4]; };      // Dirac spinor (column or row)

template <typename T> __device__ __forceinline__ R4<T> operator+(const R4<T>& a, const R4<T>& b) {
  return {{a.v[0] + b.v[0], a.v[1] + b.v[1], a.v[2] + b.v[2], a.v[3] + b.v[3]}};
}
template <typename T> __device__ __forceinline__ R4<T> operator-(const R4<T>& a) {
  return {{-a.v[0], -a.v[1], -a.v[2], -a.v[3]}};
}
template <typename T> __device__ __forceinline__ T mdot(const R4<T>& a, const R4<T>& b) {
  return fma(a.v[0], b.v[0], -fma(a.v[1], b.v[1], fma(a.v[2], b.v[2], a.v[3] * b.v[3])));
}
// Minkowski product of complex vectors (no conjugation)
template <typename T> __device__ __forceinline__ cplx<T> mdot(const V4<T>& a, const V4<T>& b) {
  cplx<T> s = a.c[0] * b.c[0];
  s = cfma(-a.c[1], b.c[1], s);
  s = cfma(-a.c[2], b.c[2], s);
  s = cfma(-a.c[3], b.c[3], s);
  return s;
}
// Minkowski product of a real with a complex vector
template <typename T> __device__ __forceinline__ cplx<T> mdot(const R4<T>& a, const V4<T>& b) {
  cplx<T> s = {a.v[0] * b.c[0].r, a.v[0] * b.c[0].i};
  s = rfma(-a.v[1], b.c[1], s);
  s = rfma(-a.v[2], b.c[2], s);
  s = rfma(-a.v[3], b.c[3], s);
  return s;
}

// ---------------------------------------------------------------------------
// gamma^mu V_mu acting on spinors.  With a = V0+V3, b = V0-V3, c = V1+iV2,
// d = V1-iV2 (complex V), the chiral-representation slash matrix is
//   [[0,0,b,-d],[0,0,-c,a],[a,d,0,0],[c,b,0,0]].
template <typename T> struct Slash { cplx<T> a, b, c, d; };

template <typename T> __device__ __forceinline__ Slash<T> make_slash(const V4<T>& V) {
  Slash<T> s;
  s.a = V.c[0] + V.c[3];
  s.b = V.c[0] - V.c[3];
  s.c = V.c[1] + times_i(V.c[2]);
  s.d = V.c[1] - times_i(V.c[2]);
  return s;
}
// (V-slash) psi for a column spinor
template <typename T> __device__ __forceinline__ S4<T> apply(const Slash<T>& s, const S4<T>& p) {
  S4<T> o;
  o.c[0] = cfma(s.b, p.c[2], -(s.d * p.c[3]));
  o.c[1] = cfma(s.a, p.c[3], -(s.c * p.c[2]));
  o.c[2] = cfma(s.a, p.c[0], s.d * p.c[1]);
  o.c[3] = cfma(s.c, p.c[0], s.b * p.c[1]);
  return o;
}
// acc += (V-slash) psi
template <typename T> __device__ __forceinline__ void apply_acc(const Slash<T>& s, const S4<T>& p, S4<T>& o) {
  o.c[0] = cfma(s.b, p.c[2], cfma(-s.d, p.c[3], o.c[0]));
  o.c[1] = cfma(s.a, p.c[3], cfma(-s.c, p.c[2], o.c[1]));
  o.c[2] = cfma(s.a, p.c[0], cfma(s.d, p.c[1], o.c[2]));
  o.c[3] = cfma(s.c, p.c[0], cfma(s.b, p.c[1], o.c[3]));
}

// Off-shell heavy-quark line with the colour-ordered factors folded in:
//   X -> -(P-slash + m) X / (P^2 - m^2 + i m Gamma)
// (the quark-gluon vertex i g gamma^mu times the propagator i(P-slash+m)/den
//  contributes i*i = -1 per step; g is factored out of the whole amplitude).
template <typename T>
__device__ __forceinline__ S4<T> quark_prop(const R4<T>& P, T m, T mw, const S4<T>& X) {
  const T a = P.v[0] + P.v[3], b = P.v[0] - P.v[3];
  const cplx<T> c = {P.v[1], P.v[2]}, d = {P.v[1], -P.v[2]};
  S4<T> y;
  y.c[0] = rfma(b, X.c[2], rfma(m, X.c[0], -(d * X.c[3])));
  y.c[1] = rfma(a, X.c[3], rfma(m, X.c[1], -(c * X.c[2])));
  y.c[2] = rfma(a, X.c[0], rfma(m, X.c[2], d * X.c[1]));
  y.c[3] = rfma(b, X.c[1], rfma(m, X.c[3], c * X.c[0]));
  const T re = mdot(P, P) - m * m;
  const T inv = T(-1) / fma(re, re, mw * mw);
  const cplx<T> f = {re * inv, -mw * inv};     // -1/den = -conj(den)/|den|^2
  S4<T> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.c[k] = y.c[k] * f;
  return o;
}

// The same with the factor f = -1/(P^2 - m^2 + i m Gamma) precomputed per
// suffix (it depends on no helicity): X -> (P-slash + m) X f.
template <typename T>
__device__ __forceinline__ S4<T> quark_prop_f(const R4<T>& P, T m, cplx<T> f, const S4<T>& X) {
  const T a = P.v[0] + P.v[3], b = P.v[0] - P.v[3];
  const cplx<T> c = {P.v[1], P.v[2]}, d = {P.v[1], -P.v[2]};
  S4<T> y;
  y.c[0] = rfma(b, X.c[2], rfma(m, X.c[0], -(d * X.c[3])));
  y.c[1] = rfma(a, X.c[3], rfma(m, X.c[1], -(c * X.c[2])));
  y.c[2] = rfma(a, X.c[0], rfma(m, X.c[2], d * X.c[1]));
  y.c[3] = rfma(b, X.c[1], rfma(m, X.c[3], c * X.c[0]));
  S4<T> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.c[k] = y.c[k] * f;
  return o;
}

template <typename T> __device__ __forceinline__ S4<T> neg(const S4<T>& a) {
  S4<T> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.c[k] = -a.c[k];
  return o;
}

template <typename T> __device__ __forceinline__ cplx<T> rowdot(const S4<T>& row, const S4<T>& col) {
  cplx<T> s = row.c[0] * col.c[0];
  s = cfma(row.c[1], col.c[1], s);
  s = cfma(row.c[2], col.c[2], s);
  s = cfma(row.c[3], col.c[3], s);
  return s;
}

// ---------------------------------------------------------------------------
// Colour-ordered gluon vertices with g factored out (P&S conventions, the
// ordered coefficient of f^{abc} T^c = -i [T^a, T^b]):
//   three-gluon (-i g) Gamma(k_L, k_R, k_out), momenta into the vertex
//   k_L = -P_L, k_R = -P_R, k_out = P_L + P_R, contracted with G_L, G_R;
//   four-gluon  (i g^2) [2 (L.R) M - (L.M) R - (M.R) L];
//   gluon propagator -i / P^2.
// Together: G(B) = [ -sum O3 + sum O4 ] / P_B^2.
template <typename T>
__device__ __forceinline__ void o3_sub(const V4<T>& GL, const V4<T>& GR, const R4<T>& PL, const R4<T>& PR, T sg,
                                       V4<T>& acc) {
  // O3 = (GL.GR)(PR - PL) - GR ((PL + 2 PR).GL) + GL ((2 PL + PR).GR); acc -= sg O3
  R4<T> a, b, c;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a.v[k] = PR.v[k] - PL.v[k];
    b.v[k] = fma(T(2), PR.v[k], PL.v[k]);
    c.v[k] = fma(T(2), PL.v[k], PR.v[k]);
  }
  const cplx<T> s0 = sg * mdot(GL, GR);
  const cplx<T> s1 = sg * mdot(b, GL);
  const cplx<T> s2 = sg * mdot(c, GR);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    cplx<T> t = rfma(-a.v[k], s0, acc.c[k]);
    t = cfma(GR.c[k], s1, t);
    acc.c[k] = cfma(-GL.c[k], s2, t);
  }
}

template <typename T>
__device__ __forceinline__ void o4_add(const V4<T>& GL, const V4<T>& GM, const V4<T>& GR, T sg, V4<T>& acc) {
  // acc += sg [2 (L.R) M - (L.M) R - (M.R) L]
  const cplx<T> lr = mdot(GL, GR), lm = sg * mdot(GL, GM), mr = sg * mdot(GM, GR);
  const cplx<T> lr2 = {T(2) * sg * lr.r, T(2) * sg * lr.i};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    cplx<T> t = cfma(lr2, GM.c[k], acc.c[k]);
    t = cfma(-lm, GR.c[k], t);
    acc.c[k] = cfma(-mr, GL.c[k], t);
  }
}

// a / b; in FP32 with the fast reciprocal (2 ulp), which is all the
// wavefunctions need
template <typename T> __device__ __forceinline__ T quot(T a, T b) { return a / b; }
template <> __device__ __forceinline__ float quot<float>(float a, float b) { return __fdividef(a, b); }

// ---------------------------------------------------------------------------
// External states.  Two-component helicity eigenstates of p/|p|:
//   chi_+ = (|p|+pz, px+i py)/sqrt(2|p|(|p|+pz)), chi_- = (-px+i py, |p|+pz)/(same),
//   limits chi_+ = (0,1), chi_- = (-1,0) along -z; +z states at rest.
template <typename T>
__device__ __forceinline__ void helicity_chi(const R4<T>& p, int lam, cplx<T>& c0, cplx<T>& c1) {
  const T px = p.v[1], py = p.v[2], pz = p.v[3];
  const T pt2 = fma(px, px, py * py);
  const T pa = sqrt(fma(pz, pz, pt2));
  // |p| + pz, free of cancellation for pz < 0: pt^2 / (|p| - pz)
  const T s = pz >= T(0) ? pa + pz : quot(pt2, pa - pz);
  if (pa == T(0)) {
    c0 = {lam > 0 ? T(1) : T(0), T(0)};
    c1 = {lam > 0 ? T(0) : T(1), T(0)};
  } else if (s > T(0)) {
    const T inv = rsqrt(T(2) * pa * s);
    if (lam > 0) { c0 = {s * inv, T(0)}; c1 = {px * inv, py * inv}; }
    else         { c0 = {-px * inv, py * inv}; c1 = {s * inv, T(0)}; }
  } else {
    if (lam > 0) { c0 = {T(0), T(0)}; c1 = {T(1), T(0)}; }
    else         { c0 = {T(-1), T(0)}; c1 = {T(0), T(0)}; }
  }
}

// omega_(+-) = sqrt(E +- |p|); omega_- = m / omega_+ (exact for an on-shell p)
template <typename T>
__device__ __forceinline__ void omegas(const R4<T>& p, T m, T& wp, T& wm) {
  const T pa = sqrt(fma(p.v[1], p.v[1], fma(p.v[2], p.v[2], p.v[3] * p.v[3])));
  wp = sqrt(p.v[0] + pa);
  wm = (m == T(0)) ? T(0) : m * rsqrt(p.v[0] + pa);
}

// ubar(p, l) for an outgoing quark: u = (w_{-l} chi_l, w_l chi_l), ubar = (u2*, u3*, u0*, u1*)
template <typename T> __device__ __forceinline__ S4<T> ubar_out(const R4<T>& p, T m, int lam) {
  T wp, wm;
  omegas(p, m, wp, wm);
  cplx<T> c0, c1;
  helicity_chi(p, lam, c0, c1);
  const T wl = lam > 0 ? wp : wm, wml = lam > 0 ? wm : wp;
  S4<T> u;
  u.c[0] = conj(wl * c0);
  u.c[1] = conj(wl * c1);
  u.c[2] = conj(wml * c0);
  u.c[3] = conj(wml * c1);
  return u;
}

// v(p, l) for an outgoing antiquark: (-l w_l chi_{-l}, l w_{-l} chi_{-l})
template <typename T> __device__ __forceinline__ S4<T> v_out(const R4<T>& p, T m, int lam) {
  T wp, wm;
  omegas(p, m, wp, wm);
  cplx<T> c0, c1;
  helicity_chi(p, -lam, c0, c1);
  const T wl = lam > 0 ? wp : wm, wml = lam > 0 ? wm : wp;
  const T sl = T(lam);
  S4<T> v;
  v.c[0] = (-sl * wl) * c0;
  v.c[1] = (-sl * wl) * c1;
  v.c[2] = (sl * wml) * c0;
  v.c[3] = (sl * wml) * c1;
  return v;
}

// Massless polarisation eps(k, l) = (-l e1 - i e2)/sqrt(2), e1/e2 along theta/phi of k
// (phi = 0 limit for k_T = 0); conjugated for an outgoing gluon.
template <typename T> __device__ __forceinline__ V4<T> polarisation(const R4<T>& k, int lam, bool outgoing) {
  const T kx = k.v[1], ky = k.v[2], kz = k.v[3];
  const T kt = sqrt(fma(kx, kx, ky * ky));
  const T ka = sqrt(fma(kt, kt, kz * kz));
  T e1[4] = {T(0), T(0), T(0), T(0)}, e2[4] = {T(0), T(0), T(0), T(0)};
  if (kt > T(0)) {
    const T ikt = T(1) / kt, ika = T(1) / ka;
    e1[1] = kx * kz * ika * ikt;
    e1[2] = ky * kz * ika * ikt;
    e1[3] = -kt * ika;
    e2[1] = -ky * ikt;
    e2[2] = kx * ikt;
  } else {
    e1[1] = kz < T(0) ? T(-1) : T(1);
    e2[2] = T(1);
  }
  const T r = T(0.70710678118654752440);
  const T sgn = outgoing ? T(1) : T(-1);       // conjugation flips the sign of the e2 part
  V4<T> e;
#pragma unroll
  for (int m = 0; m < 4; ++m) e.c[m] = {-T(lam) * r * e1[m], sgn * r * e2[m]};
  return e;
}

}  // namespace mf
