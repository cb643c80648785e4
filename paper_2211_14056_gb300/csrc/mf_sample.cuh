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

namespace mf {

constexpr int kMaxDim = 10;
constexpr int kMaxExt = 6;
constexpr double kGeV2pb = 0.3893793721e9;
constexpr double kPi = 3.14159265358979323846;

struct SampleParams {
  int n_final;          // final-state particles (2..4)
  int ndim;             // Vegas dimensions
  int nbins;            // bins per dimension
  int lumi;             // 0: fixed partonic sqrt(s); 1: synthetic gluon luminosity
  double sqrt_s;        // hadronic sqrt(S) (lumi) or partonic sqrt(s)
  double tau0, log_tau0;
  double lumi_N, lumi_a, lumi_b;
  double mt;            // top mass (final particles 0, 1 massive; gluons massless)
  double pt_cut2, dr_cut2;   // squared thresholds (0 disables)
  double phi_const;     // (2 pi)^(4-3n) (pi/2)^(n-1) / ((n-1)! (n-2)!)
};

struct EventKin {
  double p[kMaxExt][4];   // physical momenta in MadGraph order (g, g, t, tbar, g...)
  double prefactor;       // weight without |M|^2 (0 if cut / failed)
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

__device__ __forceinline__ double unit53(uint32_t a, uint32_t b) {
  const uint64_t bits = (uint64_t(a) << 21) | uint64_t(b >> 11);
  return double(bits) * 0x1.0p-53;
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

// boost p given in the rest frame of Q (mass M) into the frame of Q
__device__ __forceinline__ void boost_from_rest(const double* Q, double M, const double* p, double* out) {
  const double qp = Q[1] * p[1] + Q[2] * p[2] + Q[3] * p[3];
  const double E = (Q[0] * p[0] + qp) / M;
  const double c = (qp / (Q[0] + M) + p[0]) / M;
  out[0] = E;
  out[1] = fma(c, Q[1], p[1]);
  out[2] = fma(c, Q[2], p[2]);
  out[3] = fma(c, Q[3], p[3]);
}

// root v in [0,1] of (k+1) v^k - k v^(k+1) = r, for k = 1 (closed form) and
// k = 2 (trigonometric cubic solution), each followed by Newton polish
__device__ __forceinline__ double mass_ratio(double r, int k) {
  if (k == 1) {
    // 2v - v^2 = r  ->  v = 1 - sqrt(1 - r) = r / (1 + sqrt(1 - r))
    return r / (1.0 + sqrt(1.0 - r));
  }
  // 3 v^2 - 2 v^3 = r: v = 1/2 + cos(acos(1 - 2r)/3 - 2 pi/3)
  double v = 0.5 + cos(acos(1.0 - 2.0 * r) * (1.0 / 3.0) - 2.0943951023931954923);
  if (v < 0.0) v = 0.0;
  if (v > 1.0) v = 1.0;
  // Newton polish on f(v) = 3 v^2 - 2 v^3 - r, f' = 6 v (1 - v); restores
  // relative accuracy for small v, where the closed form cancels
  if (v <= 0.0) v = sqrt(r / 3.0);
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    const double fp = 6.0 * v * (1.0 - v);
    if (fp > 0.0) v -= (v * v * (3.0 - 2.0 * v) - r) / fp;
  }
  return v;
}

// Full per-event kinematics.  edges: [ndim][nbins+1] (shared memory).
__device__ __forceinline__ void sample_event(const SampleParams& sp, const double* edges, uint64_t seed, int iter,
                                             uint64_t ev, EventKin& out) {
  double y[kMaxDim], x[kMaxDim];
  draw_uniforms(seed, iter, ev, sp.ndim, y);
  double jac = 1.0;
  const double nb = double(sp.nbins);
  for (int j = 0; j < sp.ndim; ++j) {
    const double t = __dmul_rn(y[j], nb);
    int b = int(t);
    if (b > sp.nbins - 1) b = sp.nbins - 1;
    const double e0 = edges[j * (sp.nbins + 1) + b], e1 = edges[j * (sp.nbins + 1) + b + 1];
    const double w = e1 - e0;
    x[j] = fma(t - double(b), w, e0);
    jac *= nb * w;
    out.bins[j] = uint8_t(b);
  }
  // partonic energy and luminosity
  double shat, lum = 1.0;
  int off = 0;
  if (sp.lumi) {
    const double ua = x[0], ub = x[1];
    const double lx1 = ua * sp.log_tau0;                 // ln x1
    const double lx2 = ub * (1.0 - ua) * sp.log_tau0;    // ln x2 = ub ln(tau0/x1)
    const double x1 = exp(lx1), x2 = exp(lx2);
    shat = x1 * x2 * sp.sqrt_s * sp.sqrt_s;
    const double f1 = sp.lumi_N * exp(sp.lumi_a * lx1) * pow(1.0 - x1, sp.lumi_b);
    const double f2 = sp.lumi_N * exp(sp.lumi_a * lx2) * pow(1.0 - x2, sp.lumi_b);
    lum = f1 * f2 * x1 * x2 * (1.0 - ua) * sp.log_tau0 * sp.log_tau0;
    off = 2;
  } else {
    shat = sp.sqrt_s * sp.sqrt_s;
  }
  const double rs = sqrt(shat);
  const int n = sp.n_final;
  // RAMBO on diet: intermediate masses
  double M[kMaxExt];
  M[0] = rs;
  for (int i = 2; i <= n - 1; ++i) M[i - 1] = M[i - 2] * sqrt(mass_ratio(x[off + i - 2], n - i));
  M[n - 1] = 0.0;
  double pm[kMaxExt][4];
  double Q[4] = {rs, 0.0, 0.0, 0.0};
  double MQ = rs;
  for (int i = 1; i <= n - 1; ++i) {
    const double Mi = M[i - 1], Mn = M[i];
    const double q = (Mi - Mn) * (Mi + Mn) / (2.0 * Mi);
    const double rc = x[off + n - 2 + 2 * (i - 1)];
    const double rp = x[off + n - 2 + 2 * (i - 1) + 1];
    const double cth = 2.0 * rc - 1.0;
    const double sth = 2.0 * sqrt(rc * (1.0 - rc));
    double sph, cph;
    sincospi(2.0 * rp, &sph, &cph);
    const double pr[4] = {q, q * sth * cph, q * sth * sph, q * cth};
    const double Qr[4] = {Mi - q, -pr[1], -pr[2], -pr[3]};
    double Qn[4];
    boost_from_rest(Q, MQ, pr, pm[i - 1]);
    boost_from_rest(Q, MQ, Qr, Qn);
    for (int c = 0; c < 4; ++c) Q[c] = Qn[c];
    MQ = Mn;
  }
  for (int c = 0; c < 4; ++c) pm[n - 1][c] = Q[c];
  // Phi_n(s_hat)
  double phi = sp.phi_const;
  for (int i = 0; i < n - 2; ++i) phi *= shat;
  // massive rescaling: particles 0, 1 carry mt, the rest are massless
  const double m2 = sp.mt * sp.mt;
  double Esum = 0.0;
  for (int i = 0; i < n; ++i) Esum += pm[i][0];
  double xi = sqrt(fmax(1.0 - (2.0 * sp.mt / rs) * (2.0 * sp.mt / rs), 0.0));
  int converged = 0;
  for (int it = 0; it < 50; ++it) {
    double f = -rs, fp = 0.0;
    for (int i = 0; i < n; ++i) {
      const double E = pm[i][0];
      if (i < 2) {
        const double r = sqrt(fma(xi * E, xi * E, m2));
        f += r;
        fp += xi * E * E / r;
      } else {
        f += xi * E;
        fp += E;
      }
    }
    const double dxi = f / fp;
    xi -= dxi;
    if (fabs(dxi) <= 1e-15 * xi) { converged = 1; break; }
  }
  double ksum = 0.0, kprod = 1.0, k2sum = 0.0;
  for (int i = 0; i < n; ++i) {
    const double E = pm[i][0];
    const double k0 = (i < 2) ? sqrt(fma(xi * E, xi * E, m2)) : xi * E;
    const double ka = xi * E;      // |k| = xi |p| = xi E for massless p
    out.p[2 + i][0] = k0;
    out.p[2 + i][1] = xi * pm[i][1];
    out.p[2 + i][2] = xi * pm[i][2];
    out.p[2 + i][3] = xi * pm[i][3];
    ksum += ka;
    kprod *= ka / k0;
    k2sum += ka * ka / k0;
  }
  double wm = 1.0;
  {
    const double r = ksum / rs;
    for (int i = 0; i < 2 * n - 3; ++i) wm *= r;
    wm *= kprod * rs / k2sum;
  }
  out.p[0][0] = 0.5 * rs; out.p[0][1] = 0.0; out.p[0][2] = 0.0; out.p[0][3] = 0.5 * rs;
  out.p[1][0] = 0.5 * rs; out.p[1][1] = 0.0; out.p[1][2] = 0.0; out.p[1][3] = -0.5 * rs;
  // cuts on the final gluons (particles 4..)
  int pass = converged;
  if (sp.pt_cut2 > 0.0) {
    for (int g = 4; g < 2 + n; ++g) {
      const double pt2 = out.p[g][1] * out.p[g][1] + out.p[g][2] * out.p[g][2];
      pass &= (pt2 > sp.pt_cut2) ? 1 : 0;
    }
  }
  if (sp.dr_cut2 > 0.0) {
    for (int g = 4; g < 2 + n; ++g) {
      for (int h = g + 1; h < 2 + n; ++h) {
        const double yg = 0.5 * log((out.p[g][0] + out.p[g][3]) / (out.p[g][0] - out.p[g][3]));
        const double yh = 0.5 * log((out.p[h][0] + out.p[h][3]) / (out.p[h][0] - out.p[h][3]));
        double dphi = atan2(out.p[g][2], out.p[g][1]) - atan2(out.p[h][2], out.p[h][1]);
        if (dphi > kPi) dphi -= 2.0 * kPi;
        if (dphi < -kPi) dphi += 2.0 * kPi;
        const double dy = yg - yh;
        pass &= (dy * dy + dphi * dphi > sp.dr_cut2) ? 1 : 0;
      }
    }
  }
  out.pass = pass;
  out.newton_fail = converged ? 0 : 1;
  out.prefactor = pass ? phi * wm * jac * lum / (2.0 * shat) * kGeV2pb : 0.0;
}

}  // namespace mf
