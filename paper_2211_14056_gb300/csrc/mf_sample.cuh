// Per-event sampling: Philox uniforms -> Vegas map -> luminosity map ->
// RAMBO on diet -> massive rescaling -> cuts (one thread per event).
//
// Steps and their sources:
//  * Philox4x32-10 (Salmon et al., SC'11): key (seed_lo, seed_hi ^ iteration),
//    counter (event_lo, event_hi, dim/2, 0); dims 2j, 2j+1 take words (0,1), (2,3);
//    y = ((w_a << 21) | (w_b >> 11)) * 2^-53.
//  * Vegas map (Lepage 1978, the integrator of arXiv:2211.14056 Sec. 1):
//    bin = floor(fl(y * N_b)) clamped to N_b - 1, x = e_b + (y N_b - b)(e_{b+1} - e_b),
//    Jacobian prod N_b (e_{b+1} - e_b).  The product y * N_b is one IEEE
//    double multiply (never contracted), so bins are bit-identical to any other
//    implementation of the same definition.
//  * luminosity: x1 = tau0^u, x2 = (tau0/x1)^v, factor f(x1) f(x2) x1 x2 ln(1/tau0) ln(x1/tau0),
//    f(x) = N x^a (1-x)^b; flux 1/(2 s_hat).
//  * RAMBO on diet (Platzer, arXiv:1308.2922) with the mass-ratio equations
//    solved in closed form plus a Newton polish, then the Kleiss-Stirling-Ellis
//    massive rescaling solved by Newton in FP64 (stop at |dxi| <= 1e-15 xi,
//    at most 50 steps; a miss zeroes the weight and is counted).
//  * cuts: final-gluon pT and pairwise Delta R (dphi wrapped into [-pi, pi]).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mf_dual.cuh"
#include "mf_pdf.cuh"

namespace mf {

constexpr int kMaxDim = 10;
constexpr int kMaxExt = 6;
constexpr double kGeV2pb = 0.3893793721e9;
constexpr double kPi = 3.14159265358979323846;

struct SampleParams {
  int n_final;          // final-state particles (2..4)
  int ndim;             // Vegas dimensions
  int nbins;            // bins per dimension
  int lumi;             // 0: fixed partonic sqrt(s); 1: synthetic gluon luminosity; 2: tabulated densities
  double sqrt_s;        // hadronic sqrt(S) (lumi) or partonic sqrt(s)
  double tau0, log_tau0;
  double lumi_N, lumi_a, lumi_b;
  double mt;            // top mass (final particles 0, 1 massive; gluons and light quarks massless)
  double pt_cut2, dr_cut2;   // squared thresholds (0 disables)
  double phi_const;     // (2 pi)^(4-3n) (pi/2)^(n-1) / ((n-1)! (n-2)!)
  // lumi = 2: the set, the channel's parton pairs (flavour indices of beam 1,
  // beam 2) and ln(mu_f^2 S) (factorisation scale Q = mu_f sqrt(s_hat):
  // ln Q^2 = ln(mu_f^2 S) + ln x1 + ln x2)
  PdfView pdf;
  int npairs;
  uint8_t pairs[kMaxPdfPairs][2];
  double ln_muf2_S;
};

// K: arithmetic of the kinematics (momenta, luminosity, cuts); D: that of the
// Vegas map, the massive-rescaling Newton and the weight (FP64, or FP64 dual
// numbers in the derivative kernels).
template <typename K, typename D = double> struct EventKin {
  K p[kMaxExt][4];        // physical momenta in MadGraph order (g, g, t, tbar, g...)
  D prefactor;            // weight without |M|^2 (0 if cut / failed)
  uint8_t bins[kMaxDim];
  int pass;               // 1: compute |M|^2; 0: weight is zero
  int newton_fail;
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// m 2^-53 for the 53 bits m = (a << 21) | (b >> 11), assembled with integer
// instructions (the conversion and multiply would issue on the FP64 pipe,
// which bounds the sampler): with the leading one of m at bit p = 63 - clz(m),
// the value is 1.f 2^(p - 53), i.e. exponent field 1033 - clz(m) and the bits
// below the leading one as the fraction.  Exact, as the FP64 product is.
__device__ __forceinline__ double unit53(uint32_t a, uint32_t b) {
  const uint64_t m = (uint64_t(a) << 21) | uint64_t(b >> 11);
  if (m == 0) return 0.0;
  const int lz = __clzll((long long)m);   // 11 .. 63
  const uint64_t frac = (m << (lz - 11)) & 0x000FFFFFFFFFFFFFull;
  return __longlong_as_double((long long)((uint64_t(1033 - lz) << 52) | frac));
}

__device__ __forceinline__ void draw_uniforms(uint64_t seed, int iter, uint64_t ev, int ndim, double* y) {
  const uint2 key = make_uint2(uint32_t(seed), uint32_t(seed >> 32) ^ uint32_t(iter));
#pragma unroll
  for (int j = 0; j < (kMaxDim + 1) / 2; ++j) {
    if (2 * j < ndim) {
      const uint4 w = philox4x32_10(make_uint4(uint32_t(ev), uint32_t(ev >> 32), uint32_t(j), 0u), key);
      y[2 * j] = unit53(w.x, w.y);
      if (2 * j + 1 < ndim) y[2 * j + 1] = unit53(w.z, w.w);
    }
  }
}

// The uniform of the stream for decisions taken after the weight (the
// hit-or-miss unweighting): same key, counter (event_lo, event_hi, 0, 1),
// words (0, 1); independent of the Vegas uniforms (counters ending in 0).
__device__ __forceinline__ double unweight_uniform(uint64_t seed, int iter, uint64_t ev) {
  const uint2 key = make_uint2(uint32_t(seed), uint32_t(seed >> 32) ^ uint32_t(iter));
  const uint4 w = philox4x32_10(make_uint4(uint32_t(ev), uint32_t(ev >> 32), 0u, 1u), key);
  return unit53(w.x, w.y);
}

// boost p given in the rest frame of Q (mass M) into the frame of Q
template <typename K>
__device__ __forceinline__ void boost_from_rest(const K* Q, K M, const K* p, K* out) {
  const K qp = Q[1] * p[1] + Q[2] * p[2] + Q[3] * p[3];
  const K E = (Q[0] * p[0] + qp) / M;
  const K c = (qp / (Q[0] + M) + p[0]) / M;
  out[0] = E;
  out[1] = fma(c, Q[1], p[1]);
  out[2] = fma(c, Q[2], p[2]);
  out[3] = fma(c, Q[3], p[3]);
}

// root v in [0,1] of 3 v^2 - 2 v^3 = r: the trigonometric cubic solution,
// then Newton polish, which restores relative accuracy for small v, where the
// closed form cancels
template <typename K>
__device__ __forceinline__ K cubic_root01(K r) {
  // v = 1/2 + cos(acos(1 - 2r)/3 - 2 pi/3)
  K v = K(0.5) + cos(acos(K(1) - K(2) * r) * K(1.0 / 3.0) - K(2.0943951023931954923));
  if (v < K(0)) v = K(0);
  if (v > K(1)) v = K(1);
  // Newton on f(v) = 3 v^2 - 2 v^3 - r, f' = 6 v (1 - v)
  if (v <= K(0)) v = sqrt(r / K(3));
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    const K fp = K(6) * v * (K(1) - v);
    if (fp > K(0)) v -= (v * v * (K(3) - K(2) * v) - r) / fp;
  }
  return v;
}

// Root v in [0,1] of (k+1) v^k - k v^(k+1) = r and its complement w = 1 - v,
// from r and s = 1 - r, each given to full relative accuracy (s is formed
// before r is rounded to the kinematics type: for r within a few ulps of 1,
// 1 - r formed afterwards has no correct digit, and the two-body momentum of
// the step, M w / 2, inherits that).  k = 1: v = 1 - sqrt(s) = r / (1 +
// sqrt(s)), w = sqrt(s).  k = 2: w solves the same cubic with s in place of
// r (3 w^2 - 2 w^3 = s), so the smaller of v, w comes from its own argument.
template <typename K>
__device__ __forceinline__ void mass_ratio(K r, K s, int k, K& v, K& w) {
  if (k == 1) {
    w = sqrt(s);
    v = r / (K(1) + w);
    return;
  }
  if (r <= s) {
    v = cubic_root01(r);
    w = K(1) - v;
  } else {
    w = cubic_root01(s);
    v = K(1) - w;
  }
}

__device__ __forceinline__ void sincos_turns(double t, double* s, double* c) { sincospi(2.0 * t, s, c); }
__device__ __forceinline__ void sincos_turns(float t, float* s, float* c) { sincospif(2.0f * t, s, c); }

// Tangent seeds of the derivative kernels: tangent slot of each Vegas
// dimension's uniform and of m_t (-1: none).
struct TangentSeeds {
  int y_slot[kMaxDim];
  int mt_slot;
};

template <typename X> __device__ __forceinline__ void seed_tangent(X&, int) {}
template <typename B, int N> __device__ __forceinline__ void seed_tangent(Dual<B, N>& x, int slot) {
  if (slot >= 0 && slot < N) x.d[slot] = B(1);
}

// Full per-event kinematics.  edges: [ndim][nbins+1] (shared memory).
// K = double: every step in FP64.  K = float: luminosity, RAMBO and cuts in
// FP32; bins, map, Jacobian, Newton (polished to 1e-15 in FP64) and weight in
// FP64.  D = dual numbers: the same steps carry tangents seeded by ts.
// Every loop over dimensions or particles runs to the compile-time maximum
// (kMaxDim, kMaxExt) behind a guard on the runtime count, fully unrolled, so
// that every per-particle and per-dimension array is indexed by constants and
// lives in registers (a runtime index would put them in local memory).
template <typename K, typename D = double>
__device__ __forceinline__ void sample_event(const SampleParams& sp, const double* edges, uint64_t seed, int iter,
                                             uint64_t ev, EventKin<K, D>& out, const TangentSeeds* ts = nullptr) {
  double y[kMaxDim];
  D x[kMaxDim];
  const int ndim = sp.ndim;
  draw_uniforms(seed, iter, ev, ndim, y);
  double jac = 1.0;
  const double nb = double(sp.nbins);
#pragma unroll
  for (int j = 0; j < kMaxDim; ++j) {
    if (j < ndim) {
      const double t = __dmul_rn(y[j], nb);
      int b = int(t);
      if (b > sp.nbins - 1) b = sp.nbins - 1;
      const double e0 = edges[j * (sp.nbins + 1) + b], e1 = edges[j * (sp.nbins + 1) + b + 1];
      const double w = e1 - e0;
      if constexpr (is_dual<D>::value) {
        D yd = D(y[j]);
        if (ts) seed_tangent(yd, ts->y_slot[j]);
        x[j] = (yd * nb - double(b)) * w + e0;
      } else {
        x[j] = fma(t - double(b), w, e0);
      }
      jac *= nb * w;
      out.bins[j] = uint8_t(b);
    } else {
      x[j] = D(0.0);
      out.bins[j] = 0;
    }
  }
  D mtd = D(sp.mt);
  if (ts) seed_tangent(mtd, ts->mt_slot);
  // partonic energy and luminosity
  D shat, lum = D(1.0), excess;
  const D thr = D(2.0) * mtd;
  if (sp.lumi) {
    // ln x1 = u ln tau0, ln x2 = v (1 - u) ln tau0 (= v ln(tau0/x1));
    // f(x1) f(x2) x1 x2 = N^2 exp((a + 1)(ln x1 + ln x2) + b (ln(1-x1) + ln(1-x2)))
    D log_tau0;
    if constexpr (is_dual<D>::value) log_tau0 = log(thr * thr / D(sp.sqrt_s * sp.sqrt_s));
    else log_tau0 = sp.log_tau0;
    const K lt = K(log_tau0);
    const K lx[2] = {K(x[0]) * lt, K(x[1]) * (K(1) - K(x[0])) * lt};
    // ln(1 - x) = ln(-expm1(ln x)): accurate also for x within an ulp of 1
    // (where 1 - exp(ln x) would round to 0 in FP32)
    const K lsum = lx[0] + lx[1];
    shat = D(exp(lsum)) * (sp.sqrt_s * sp.sqrt_s);
    if (sp.lumi == 2) {
      // tabulated densities: sum over the channel's parton pairs of
      // x1 f_a(x1, Q^2) x2 f_b(x2, Q^2) (the map's x1 x2 is in the table's x f)
      // (the derivative pass does not cover tabulated densities: no tangents here)
      K L = K(0);
      if constexpr (!is_dual<K>::value) {
        const K lq2 = K(sp.ln_muf2_S) + lsum;
        const PdfCell<K> c1 = pdf_cell(sp.pdf, lx[0], lq2), c2 = pdf_cell(sp.pdf, lx[1], lq2);
#pragma unroll 1
        for (int k = 0; k < sp.npairs; ++k)
          L += pdf_xfx(sp.pdf, sp.pairs[k][0], c1) * pdf_xfx(sp.pdf, sp.pairs[k][1], c2);
      }
      lum = D(L) * (D(1.0) - x[0]) * log_tau0 * log_tau0;
    } else {
      const K l1m = log(-expm1(lx[0])) + log(-expm1(lx[1]));
      const K ff = exp(K(sp.lumi_a + 1.0) * lsum + K(sp.lumi_b) * l1m);
      lum = D(ff) * (D(1.0) - x[0]) * log_tau0 * log_tau0 * (sp.lumi_N * sp.lumi_N);
    }
  } else {
    shat = D(sp.sqrt_s * sp.sqrt_s);
  }
  // the phase-space uniforms: the dimensions after the luminosity's two
  D xr[kMaxDim - 2];
#pragma unroll
  for (int j = 0; j < kMaxDim - 2; ++j) xr[j] = sp.lumi ? x[j + 2] : x[j];
  const D rs = sqrt(shat);
  const K rsk = K(rs);
  const int n = sp.n_final;
  // RAMBO on diet: intermediate masses M[i - 1] of Q_i (M[0] = sqrt(s_hat),
  // M[n - 1] = 0) and the complements W[i - 1] = 1 - M[i]^2 / M[i - 1]^2 of
  // their squared ratios (W = 1 at the last step)
  K M[kMaxExt], W[kMaxExt];
  M[0] = rsk;
#pragma unroll
  for (int i = 2; i <= kMaxExt; ++i) {
    W[i - 2] = K(1);
    if (i <= n - 1) {
      K v, wc;
      mass_ratio(K(xr[i - 2]), K(D(1.0) - xr[i - 2]), n - i, v, wc);
      M[i - 1] = M[i - 2] * sqrt(v);
      W[i - 2] = wc;
    } else {
      M[i - 1] = K(0);
    }
  }
  W[kMaxExt - 1] = K(1);
  // the angle uniforms xa: the phase-space uniforms after the n - 2 mass
  // ones, shifted one place per mass uniform (a runtime offset into xr would
  // be a runtime index)
  D xa[kMaxDim - 2];
#pragma unroll
  for (int j = 0; j < kMaxDim - 2; ++j) xa[j] = xr[j];
#pragma unroll
  for (int s = 0; s < kMaxExt - 2; ++s)
    if (s < n - 2)
#pragma unroll
      for (int j = 0; j < kMaxDim - 3; ++j) xa[j] = xa[j + 1];
  K pm[kMaxExt][4];
  K Q[4] = {rsk, K(0), K(0), K(0)};
  K MQ = rsk;
#pragma unroll
  for (int i = 1; i <= kMaxExt - 1; ++i) {
    if (i <= n - 1) {
      const K Mi = M[i - 1], Mn = M[i];
      // massless momentum of the two-body step, (Mi^2 - Mn^2) / (2 Mi), as
      // Mi (1 - Mn^2/Mi^2) / 2 with the accurate complement
      const K q = K(0.5) * Mi * W[i - 1];
      // (cos theta, phi) uniforms of this step: after the n - 2 mass uniforms;
      // sin theta from rc (1 - rc) with 1 - rc formed before rounding
      const K rc = K(xa[2 * (i - 1)]), rcm = K(D(1.0) - xa[2 * (i - 1)]), rp = K(xa[2 * (i - 1) + 1]);
      const K cth = rc - rcm;
      const K sth = K(2) * sqrt(rc * rcm);
      K sph, cph;
      sincos_turns(rp, &sph, &cph);
      const K pr[4] = {q, q * sth * cph, q * sth * sph, q * cth};
      const K Qr[4] = {Mi - q, -pr[1], -pr[2], -pr[3]};
      K Qn[4];
      boost_from_rest(Q, MQ, pr, pm[i - 1]);
      boost_from_rest(Q, MQ, Qr, Qn);
      // Q_{i+1}; after the last step it is the last massless momentum (a
      // later step, if any, overwrites pm[i] with its own decay product)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        Q[c] = Qn[c];
        pm[i][c] = Qn[c];
      }
      MQ = Mn;
    }
  }
  // Phi_n(s_hat)
  D phi = D(sp.phi_const);
  for (int i = 0; i < n - 2; ++i) phi = phi * shat;
  // f(xi) = sum_{i=0,1} (sqrt(m^2 + xi^2 E_i^2) - m) + xi E_rest - (sqrt(s) - 2m), with
  // sqrt(m^2 + u^2) - m = u^2 / (sqrt(m^2 + u^2) + m): no cancellation near
  // threshold, so Newton reaches full relative precision in xi there too.
  // Stop after a step |dxi| <= tol xi: f is convex with xi f''/f' =
  // sum m^2 E^2 xi / r^3 / (sum xi E^2 / r + E_rest) <= 1 (m <= r), so a
  // Newton step of relative size d from that close leaves a relative error
  // below d^2 / 2: tol = 1e-8 (5e-17) for FP64 kinematics; 1e-6 (5e-13,
  // far below the FP32 momenta's rounding) for FP32 kinematics, where the
  // first FP64 step from the converged FP32 start (relative size ~1e-7)
  // already meets it; 50 steps at most.  With dual numbers the
  // converged xi is refined by one more step, which carries the
  // implicit-function derivative d xi = -(df/dtheta) / f'.
  const D m2 = mtd * mtd;
  D E[kMaxExt];
  D Erest = D(0.0);
#pragma unroll
  for (int i = 0; i < kMaxExt; ++i) {
    if (i < n) {
      E[i] = D(pm[i][0]);
      if (i >= 2) Erest = Erest + E[i];
    } else {
      E[i] = D(0.0);
    }
  }
  excess = (shat - thr * thr) / (rs + thr);     // sqrt(s) - 2m
  const D irs = D(1.0) / rs;                     // one FP64 division for the three uses below
  double xi0 = sqrt(fmax(value_of(excess) * value_of(rs + thr), 0.0)) * value_of(irs);
  if constexpr (sizeof(value_of(K(0))) < sizeof(double)) {
    using KB = decltype(value_of(K(0)));
    const KB m2k = KB(value_of(m2)), mk = KB(value_of(mtd)), e0 = value_of(pm[0][0]), e1 = value_of(pm[1][0]),
             er = KB(value_of(Erest)), exk = KB(value_of(excess));
    KB xk = KB(xi0);
#pragma unroll 1
    for (int it = 0; it < 20; ++it) {
      const KB u0 = xk * e0, u1 = xk * e1;
      const KB r0 = sqrt(fma(u0, u0, m2k)), r1 = sqrt(fma(u1, u1, m2k));
      const KB f = u0 * u0 / (r0 + mk) + u1 * u1 / (r1 + mk) + xk * er - exk;
      const KB fp = xk * (e0 * e0 / r0 + e1 * e1 / r1) + er;
      const KB d = f / fp;
      xk -= d;
      if (fabs(d) <= KB(1e-6) * xk) break;
    }
    if (xk > KB(0) && xk < KB(1)) xi0 = double(xk);
  }
  int converged = 0;
  {
    const double mv = value_of(mtd), m2v = value_of(m2), e0 = value_of(E[0]), e1 = value_of(E[1]);
    const double er = value_of(Erest), exv = value_of(excess);
    constexpr double tol = sizeof(value_of(K(0))) < sizeof(double) ? 1e-6 : 1e-8;
    double xi = xi0;
#pragma unroll 1
    for (int it = 0; it < 50; ++it) {
      const double u0 = xi * e0, u1 = xi * e1;
      const double r0 = sqrt(fma(u0, u0, m2v)), r1 = sqrt(fma(u1, u1, m2v));
      // the four fractions over one common denominator (one division; every
      // term is positive, so nothing cancels)
      const double A = r0 + mv, B = r1 + mv, rr = r0 * r1, ab = A * B;
      const double iden = 1.0 / (ab * rr);
      const double f = fma(u0 * u0, B, u1 * u1 * A) * rr * iden + fma(xi, er, -exv);
      const double fp = fma(xi * fma(e0 * e0, r1, e1 * e1 * r0), ab * iden, er);
      const double dxi = f / fp;
      xi -= dxi;
      if (fabs(dxi) <= tol * xi) { converged = 1; break; }
    }
    xi0 = xi;
  }
  D xi = D(xi0);
  if constexpr (is_dual<D>::value) {
    const D u0 = xi * E[0], u1 = xi * E[1];
    const D r0 = sqrt(u0 * u0 + m2), r1 = sqrt(u1 * u1 + m2);
    const D f = u0 * u0 / (r0 + mtd) + u1 * u1 / (r1 + mtd) + xi * Erest - excess;
    const D fp = xi * (E[0] * E[0] / r0 + E[1] * E[1] / r1) + Erest;
    xi = xi - f / fp;
  }
  // |k| = xi |p| = xi E for massless p; the massless final particles have
  // |k| / k0 = 1, so only the two massive ones enter the product, over one
  // common denominator
  const D ka0 = xi * E[0], ka1 = xi * E[1];
  const D k00 = sqrt(ka0 * ka0 + m2), k01 = sqrt(ka1 * ka1 + m2);
  const D ik = D(1.0) / (k00 * k01);
  const D kprod = ka0 * ka1 * ik;
  D ksum = ka0 + ka1, k2sum = (ka0 * ka0 * k01 + ka1 * ka1 * k00) * ik;
  out.p[2][0] = K(k00);
  out.p[3][0] = K(k01);
#pragma unroll
  for (int i = 0; i < kMaxExt - 2; ++i) {
    if (i < n) {
      if (i >= 2) {
        const D ka = xi * E[i];
        out.p[2 + i][0] = K(ka);
        ksum = ksum + ka;
        k2sum = k2sum + ka;
      }
      if constexpr (std::is_same<K, float>::value && std::is_same<D, double>::value) {
        // FP32 kinematics: the massless components are FP32; scaling them in
        // FP32 (one more rounding, 1.2e-7 at most) saves two FP64-pipe
        // conversions and a multiply per component
        const float xf = float(xi);
        out.p[2 + i][1] = xf * pm[i][1];
        out.p[2 + i][2] = xf * pm[i][2];
        out.p[2 + i][3] = xf * pm[i][3];
      } else {
        out.p[2 + i][1] = K(xi * D(pm[i][1]));
        out.p[2 + i][2] = K(xi * D(pm[i][2]));
        out.p[2 + i][3] = K(xi * D(pm[i][3]));
      }
    }
  }
  D wm = D(1.0);
  {
    const D r = ksum * irs;
    for (int i = 0; i < 2 * n - 3; ++i) wm = wm * r;
    wm = wm * (kprod * rs / k2sum);
  }
  const K hr = K(D(0.5) * rs);
  out.p[0][0] = hr; out.p[0][1] = K(0); out.p[0][2] = K(0); out.p[0][3] = hr;
  out.p[1][0] = hr; out.p[1][1] = K(0); out.p[1][2] = K(0); out.p[1][3] = -hr;
  // cuts on the final gluons (particles 4..)
  int pass = converged;
  if (sp.pt_cut2 > 0.0) {
#pragma unroll
    for (int g = 4; g < kMaxExt; ++g) {
      if (g < 2 + n) {
        const K pt2 = out.p[g][1] * out.p[g][1] + out.p[g][2] * out.p[g][2];
        pass &= (pt2 > K(sp.pt_cut2)) ? 1 : 0;
      }
    }
  }
  if (sp.dr_cut2 > 0.0) {
    // Delta y = ln[(E_g + z_g)(E_h - z_h) / ((E_g - z_g)(E_h + z_h))] / 2,
    // Delta phi = atan2(cross, dot) of the transverse momenta (in [-pi, pi])
#pragma unroll
    for (int g = 4; g < kMaxExt; ++g) {
#pragma unroll
      for (int h = g + 1; h < kMaxExt; ++h) {
        if (h < 2 + n) {
          const K dy = K(0.5) * log(((out.p[g][0] + out.p[g][3]) * (out.p[h][0] - out.p[h][3])) /
                                    ((out.p[g][0] - out.p[g][3]) * (out.p[h][0] + out.p[h][3])));
          const K cr = out.p[g][1] * out.p[h][2] - out.p[g][2] * out.p[h][1];
          const K dt = out.p[g][1] * out.p[h][1] + out.p[g][2] * out.p[h][2];
          const K dphi = atan2(cr, dt);
          pass &= (dy * dy + dphi * dphi > K(sp.dr_cut2)) ? 1 : 0;
        }
      }
    }
  }
  out.pass = pass;
  out.newton_fail = converged ? 0 : 1;
  out.prefactor = pass ? phi * wm * lum * (D(0.5) * irs * irs) * (jac * kGeV2pb) : D(0.0);
}

}  // namespace mf
