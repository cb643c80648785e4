"""Phase space: RAMBO on diet, massive rescaling, classic RAMBO, luminosity, cuts.

Test infrastructure (see ``oracle/__init__``).

The paper (arXiv:2211.14056) does not spell out its phase-space generator; the
hot path uses these published algorithms:

* RAMBO on diet (S. Platzer, arXiv:1308.2922): n massless momenta with total
  momentum (sqrt(s), 0) from 3n-4 uniforms and the constant weight
      Phi_n = (2 pi)^(4-3n) (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!).
  Intermediate masses M_1 = sqrt(s) > M_2 > ... > M_n = 0 follow from
  M_i = M_(i-1) sqrt(v_i), where v_i solves
      r_i = (n+1-i) v^(n-i) - (n-i) v^(n+1-i),   i = 2..n-1,
  and each Q_i (mass M_i) decays isotropically into a massless p_i and Q_(i+1).
  Uniform order: the n-2 mass uniforms, then (cos theta, phi) pairs.
* Massive rescaling (R. Kleiss, W.J. Stirling, S.D. Ellis, CPC 40 (1986) 359):
  solve sum_i sqrt(m_i^2 + xi^2 E_i^2) = sqrt(s) for xi, set
  k_i = (sqrt(m_i^2 + xi^2 E_i^2), xi p_i) and multiply the weight by
      (sum|k|/sqrt s)^(2n-3) prod(|k_i|/k_i^0) sqrt(s) / sum(|k_i|^2/k_i^0).
* Classic RAMBO (same CPC paper), used only to test the diet version.
* Synthetic gluon luminosity f(x) = N x^a (1-x)^b with the map
  x1 = tau0^u, x2 = (tau0/x1)^v, tau0 = 4 m_t^2 / S, Jacobian
  x1 x2 ln(1/tau0) ln(x1/tau0); flux 1/(2 s_hat).
* Cuts: gluon pT and pairwise Delta R = sqrt(dy^2 + dphi^2), dphi in [-pi, pi].

Momenta are arrays [N, n, 4] with components (E, px, py, pz).
"""
import math
import numpy as np

GEV2_TO_PB = 0.3893793721e9


def massless_volume(n, s):
    """Phi_n(s) of n massless particles (RAMBO on diet normalisation)."""
    return ((2 * math.pi) ** (4 - 3 * n) * (math.pi / 2) ** (n - 1) * s ** (n - 2)
            / (math.factorial(n - 1) * math.factorial(n - 2)))


def boost_from_rest(p, Q):
    """Boost p (given in the rest frame of Q) to the frame where Q is given.

    p, Q: [..., 4].  Standard pure boost with velocity Q_vec / Q_0.
    """
    M = np.sqrt(np.maximum(Q[..., 0] ** 2 - np.sum(Q[..., 1:] ** 2, axis=-1), 0.0))
    qp = np.sum(Q[..., 1:] * p[..., 1:], axis=-1)
    E = (Q[..., 0] * p[..., 0] + qp) / M
    c = (qp / (Q[..., 0] + M) + p[..., 0]) / M
    out = np.empty_like(p)
    out[..., 0] = E
    out[..., 1:] = p[..., 1:] + c[..., None] * Q[..., 1:]
    return out


def _solve_mass_ratio(r, n, i, iters=200):
    """Root v in [0, 1] of (n+1-i) v^(n-i) - (n-i) v^(n+1-i) = r, by bisection.

    The left side rises monotonically from 0 at v = 0 to 1 at v = 1.
    """
    lo = np.zeros_like(r)
    hi = np.ones_like(r)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        f = (n + 1 - i) * mid ** (n - i) - (n - i) * mid ** (n + 1 - i) - r
        below = f < 0
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
        if np.all(hi - lo <= 0):
            break
    return 0.5 * (lo + hi)


def rambo_diet(sqrt_s, r, n):
    """n massless momenta [N, n, 4] in the CM frame from uniforms r[3n-4, N].

    sqrt_s may be a scalar or an array [N].  Returns (p, weight[N]).
    """
    r = np.asarray(r, dtype=np.float64)
    N = r.shape[1]
    sqrt_s = np.broadcast_to(np.asarray(sqrt_s, dtype=np.float64), (N,))
    M = [sqrt_s]
    for i in range(2, n):
        v = _solve_mass_ratio(r[i - 2], n, i)
        M.append(M[-1] * np.sqrt(v))
    M.append(np.zeros(N))
    p = np.empty((N, n, 4))
    Q = np.zeros((N, 4))
    Q[:, 0] = sqrt_s
    for i in range(1, n):
        Mi, Mn = M[i - 1], M[i]
        q = (Mi * Mi - Mn * Mn) / (2.0 * Mi)
        cos_t = 2.0 * r[n - 2 + 2 * (i - 1)] - 1.0
        phi = 2.0 * math.pi * r[n - 2 + 2 * (i - 1) + 1]
        sin_t = np.sqrt(np.maximum(1.0 - cos_t * cos_t, 0.0))
        pr = np.stack([q, q * sin_t * np.cos(phi), q * sin_t * np.sin(phi), q * cos_t], axis=-1)
        Qr = np.stack([Mi - q, -pr[:, 1], -pr[:, 2], -pr[:, 3]], axis=-1)
        p[:, i - 1] = boost_from_rest(pr, Q)
        Q = boost_from_rest(Qr, Q)
    p[:, n - 1] = Q
    w = np.array([massless_volume(n, s) for s in sqrt_s ** 2])
    return p, w


def rambo_classic(sqrt_s, r, n):
    """Classic RAMBO: n massless momenta from 4n uniforms r[4n, N] (CPC 40)."""
    N = r.shape[1]
    q = np.empty((N, n, 4))
    for i in range(n):
        c = 2.0 * r[4 * i] - 1.0
        s = np.sqrt(1.0 - c * c)
        f = 2.0 * math.pi * r[4 * i + 1]
        e = -np.log(r[4 * i + 2] * r[4 * i + 3])
        q[:, i] = np.stack([e, e * s * np.cos(f), e * s * np.sin(f), e * c], axis=-1)
    Q = q.sum(axis=1)
    M = np.sqrt(Q[:, 0] ** 2 - np.sum(Q[:, 1:] ** 2, axis=-1))
    b = -Q[:, 1:] / M[:, None]
    x = sqrt_s / M
    gam = Q[:, 0] / M
    a = 1.0 / (1.0 + gam)
    p = np.empty_like(q)
    for i in range(n):
        bq = np.sum(b * q[:, i, 1:], axis=-1)
        p[:, i, 0] = x * (gam * q[:, i, 0] + bq)
        p[:, i, 1:] = x[:, None] * (q[:, i, 1:] + b * q[:, i, 0][:, None] + (a * bq)[:, None] * b)
    return p, np.full(N, massless_volume(n, sqrt_s ** 2))


def solve_xi(E, masses, sqrt_s, iters=200):
    """xi in [0, 1] with sum_i sqrt(m_i^2 + xi^2 E_i^2) = sqrt(s), by bisection.

    E: [N, n] massless energies summing to sqrt(s).
    """
    m2 = np.asarray(masses, dtype=np.float64) ** 2
    lo = np.zeros(E.shape[0])
    hi = np.ones(E.shape[0])
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        f = np.sum(np.sqrt(m2[None, :] + (mid[:, None] * E) ** 2), axis=1) - sqrt_s
        below = f < 0
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


def massive(p, masses, sqrt_s):
    """Kleiss-Stirling-Ellis rescaling of massless p [N, n, 4] to the masses.

    Returns (k [N, n, 4], weight factor [N]).
    """
    n = p.shape[1]
    sqrt_s = np.broadcast_to(np.asarray(sqrt_s, dtype=np.float64), (p.shape[0],))
    m = np.asarray(masses, dtype=np.float64)
    E = p[:, :, 0]
    xi = solve_xi(E, m, sqrt_s)
    k = np.empty_like(p)
    k[:, :, 1:] = xi[:, None, None] * p[:, :, 1:]
    k[:, :, 0] = np.sqrt(m[None, :] ** 2 + (xi[:, None] * E) ** 2)
    kabs = np.sqrt(np.sum(k[:, :, 1:] ** 2, axis=-1))
    w = ((np.sum(kabs, axis=1) / sqrt_s) ** (2 * n - 3) * np.prod(kabs / k[:, :, 0], axis=1)
         * sqrt_s / np.sum(kabs ** 2 / k[:, :, 0], axis=1))
    return k, w


def luminosity_map(ua, ub, tau0, S, N=1.0, a=-1.1, b=5.0):
    """(x1, x2, s_hat, factor): f(x1) f(x2) times the map's Jacobian.

    f(x) = N x^a (1-x)^b, x1 = tau0^ua, x2 = (tau0/x1)^ub.
    """
    x1 = tau0 ** ua
    x2 = (tau0 / x1) ** ub
    f = lambda x: N * x ** a * (1.0 - x) ** b
    jac = x1 * x2 * math.log(1.0 / tau0) * np.log(x1 / tau0)
    return x1, x2, x1 * x2 * S, f(x1) * f(x2) * jac


def pdf_luminosity_map(ua, ub, tau0, S, pdf, pairs, mu_f):
    """(x1, x2, s_hat, factor) with tabulated parton densities: the same map
    as ``luminosity_map``; the factor is sum over the parton pairs (a, b) of
    x1 f_a(x1, Q^2) x2 f_b(x2, Q^2) (the map's x1 x2 absorbed into the
    tabulated x f) times ln(1/tau0) ln(x1/tau0), at the factorisation scale
    Q = mu_f sqrt(s_hat).  pdf: an ``oracle.pdf.PDFGrid``."""
    x1 = tau0 ** ua
    x2 = (tau0 / x1) ** ub
    shat = x1 * x2 * S
    q2 = mu_f * mu_f * shat
    lum = 0.0
    for a, b in pairs:
        lum = lum + pdf.xfx(a, x1, q2) * pdf.xfx(b, x2, q2)
    return x1, x2, shat, lum * math.log(1.0 / tau0) * np.log(x1 / tau0)


def pt(p):
    return np.sqrt(p[..., 1] ** 2 + p[..., 2] ** 2)


def rapidity(p):
    return 0.5 * np.log((p[..., 0] + p[..., 3]) / (p[..., 0] - p[..., 3]))


def delta_r(p, q):
    dy = rapidity(p) - rapidity(q)
    dphi = np.arctan2(p[..., 2], p[..., 1]) - np.arctan2(q[..., 2], q[..., 1])
    dphi = (dphi + math.pi) % (2 * math.pi) - math.pi
    return np.sqrt(dy * dy + dphi * dphi)


def pass_cuts(k, gluons, pt_min, dr_min):
    """Boolean [N]: every listed final gluon has pT > pt_min and every pair
    of them Delta R > dr_min (a zero threshold disables that cut)."""
    ok = np.ones(k.shape[0], dtype=bool)
    if pt_min > 0:
        for g in gluons:
            ok &= pt(k[:, g]) > pt_min
    if dr_min > 0:
        for i, g in enumerate(gluons):
            for h in gluons[i + 1:]:
                ok &= delta_r(k[:, g], k[:, h]) > dr_min
    return ok
