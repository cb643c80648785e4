// Primitives of the u u~ -> t t~ g g amplitude (Feynman-diagram form, see
// gen_uux.py): external light-quark spinors, row and column slashes, light
// and heavy quark propagators, the vector current of a fermion line, the
// gluon propagator and the three- and four-gluon Lorentz structures
// (Peskin-Schroeder vertices with the coupling and the factors of i taken out;
// the generated code multiplies each diagram by its power of i).
#pragma once
#include "mf_device.cuh"

namespace mf {

// u(p, l) of an incoming quark: (w_{-l} chi_l, w_l chi_l)
template <typename T> __device__ __forceinline__ S4<T> u_in(const R4<T>& p, T m, int lam) {
  T wp, wm;
  omegas(p, m, wp, wm);
  cplx<T> c0, c1;
  helicity_chi(p, lam, c0, c1);
  const T wl = lam > 0 ? wp : wm, wml = lam > 0 ? wm : wp;
  S4<T> u;
  u.c[0] = wml * c0;
  u.c[1] = wml * c1;
  u.c[2] = wl * c0;
  u.c[3] = wl * c1;
  return u;
}

// vbar(p, l) of an incoming antiquark: v = (-l w_l chi_{-l}, l w_{-l} chi_{-l}),
// vbar = v^dagger gamma^0 = (v2*, v3*, v0*, v1*)
template <typename T> __device__ __forceinline__ S4<T> vbar_in(const R4<T>& p, T m, int lam) {
  const S4<T> v = v_out(p, m, lam);
  S4<T> r;
  r.c[0] = conj(v.c[2]);
  r.c[1] = conj(v.c[3]);
  r.c[2] = conj(v.c[0]);
  r.c[3] = conj(v.c[1]);
  return r;
}

// row spinor times V-slash
template <typename T> __device__ __forceinline__ S4<T> slash_row(const S4<T>& R, const V4<T>& V) {
  const Slash<T> s = make_slash(V);
  S4<T> o;
  o.c[0] = cfma(R.c[2], s.a, R.c[3] * s.c);
  o.c[1] = cfma(R.c[2], s.d, R.c[3] * s.b);
  o.c[2] = cfma(R.c[0], s.b, -(R.c[1] * s.c));
  o.c[3] = cfma(R.c[1], s.a, -(R.c[0] * s.d));
  return o;
}

template <typename T> __device__ __forceinline__ V4<T> real_vec(const R4<T>& P) {
  V4<T> v;
#pragma unroll
  for (int k = 0; k < 4; ++k) v.c[k] = {P.v[k], T(0)};
  return v;
}

// massless propagator numerator and denominator: P-slash X / P^2
template <typename T> __device__ __forceinline__ S4<T> lprop_col(const R4<T>& P, const S4<T>& X) {
  const T inv = T(1) / mdot(P, P);
  S4<T> y = apply(make_slash(real_vec(P)), X);
#pragma unroll
  for (int k = 0; k < 4; ++k) y.c[k] = inv * y.c[k];
  return y;
}

template <typename T> __device__ __forceinline__ S4<T> lprop_row(const S4<T>& R, const R4<T>& P) {
  const T inv = T(1) / mdot(P, P);
  S4<T> y = slash_row(R, real_vec(P));
#pragma unroll
  for (int k = 0; k < 4; ++k) y.c[k] = inv * y.c[k];
  return y;
}

// heavy propagator: (P-slash + m) X / (P^2 - m^2 + i m Gamma)
template <typename T> __device__ __forceinline__ S4<T> hprop_col(const R4<T>& P, T m, T mw, const S4<T>& X) {
  const T re = mdot(P, P) - m * m;
  const T inv = T(1) / fma(re, re, mw * mw);
  const cplx<T> f = {re * inv, -mw * inv};        // 1/(re + i mw)
  S4<T> y = apply(make_slash(real_vec(P)), X);
  S4<T> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.c[k] = rfma(m, X.c[k], y.c[k]) * f;
  return o;
}

// L^mu = R gamma^mu C (chiral representation): with the slash coefficients
// a = V0+V3, b = V0-V3, c = V1+iV2, d = V1-iV2 of R V-slash C
template <typename T> __device__ __forceinline__ V4<T> vcur(const S4<T>& R, const S4<T>& C) {
  const cplx<T> ca = cfma(R.c[1], C.c[3], R.c[2] * C.c[0]);
  const cplx<T> cb = cfma(R.c[0], C.c[2], R.c[3] * C.c[1]);
  const cplx<T> cc = cfma(R.c[3], C.c[0], -(R.c[1] * C.c[2]));
  const cplx<T> cd = cfma(R.c[2], C.c[1], -(R.c[0] * C.c[3]));
  V4<T> L;
  L.c[0] = ca + cb;
  L.c[1] = -(cc + cd);
  L.c[2] = times_i(cd - cc);     // -i (cc - cd)
  L.c[3] = cb - ca;
  return L;
}

// gluon propagator (g_mu_nu and -i taken out): V / K^2
template <typename T> __device__ __forceinline__ V4<T> gprop(const V4<T>& V, const R4<T>& K) {
  const T inv = T(1) / mdot(K, K);
  V4<T> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.c[k] = inv * V.c[k];
  return o;
}

// three-gluon structure contracted with A (momentum KA into the vertex) and
// C (KC): (A.C)(KA - KC) + C ((KA + 2 KC).A) - A ((2 KA + KC).C)
template <typename T>
__device__ __forceinline__ V4<T> vvv(const V4<T>& A, const R4<T>& KA, const V4<T>& C, const R4<T>& KC) {
  R4<T> d, e, f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    d.v[k] = KA.v[k] - KC.v[k];
    e.v[k] = fma(T(2), KC.v[k], KA.v[k]);
    f.v[k] = fma(T(2), KA.v[k], KC.v[k]);
  }
  const cplx<T> s0 = mdot(A, C), s1 = mdot(e, A), s2 = mdot(f, C);
  V4<T> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.c[k] = cfma(C.c[k], s1, cfma(-A.c[k], s2, d.v[k] * s0));
  return o;
}

// four-gluon structures for the colour terms f^abe f^cde (1), f^ace f^bde (2),
// f^ade f^bce (3) with A, C, D on legs a, b, c
template <int TERM, typename T>
__device__ __forceinline__ V4<T> v4_term(const V4<T>& A, const V4<T>& C, const V4<T>& D) {
  V4<T> o;
  if constexpr (TERM == 1) {
    const cplx<T> ad = mdot(A, D), cd = mdot(C, D);
#pragma unroll
    for (int k = 0; k < 4; ++k) o.c[k] = cfma(ad, C.c[k], -(cd * A.c[k]));
  } else if constexpr (TERM == 2) {
    const cplx<T> ac = mdot(A, C), cd = mdot(C, D);
#pragma unroll
    for (int k = 0; k < 4; ++k) o.c[k] = cfma(ac, D.c[k], -(cd * A.c[k]));
  } else {
    const cplx<T> ac = mdot(A, C), ad = mdot(A, D);
#pragma unroll
    for (int k = 0; k < 4; ++k) o.c[k] = cfma(ac, D.c[k], -(ad * C.c[k]));
  }
  return o;
}

}  // namespace mf
