"""Pins for oracle.phase_space.

* RAMBO on diet: momentum conservation, masslessness, the closed-form volume
  Phi_n (Phi_2 = 1/(8 pi)), and the distributions of all pair invariants equal
  to classic RAMBO's (two-sample KS);
* massive rescaling: on-shell masses, conservation, the two-body weight
  beta/(8 pi) exactly, and the three-body mean weight equal to the Dalitz
  volume (1/(128 pi^3 s)) * area, the area from 1-D quadrature;
* luminosity map: x1 x2 >= tau0 and the Jacobian by finite differences;
* cuts on hand-built momenta.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import phase_space as ps


def mdot(a, b):
    return a[..., 0] * b[..., 0] - np.sum(a[..., 1:] * b[..., 1:], axis=-1)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_rambo_diet_conservation_and_volume(n):
    rng = np.random.default_rng(n)
    rs = 1234.5
    p, w = ps.rambo_diet(rs, rng.random((3 * n - 4, 2000)), n)
    tot = p.sum(axis=1)
    # boosts out of light intermediate masses lose a few digits (gamma ~ 1e3)
    np.testing.assert_allclose(tot[:, 0], rs, rtol=1e-11)
    np.testing.assert_allclose(tot[:, 1:], 0, atol=1e-11 * rs)
    np.testing.assert_allclose(mdot(p, p), 0, atol=1e-11 * rs * rs)
    assert np.all(p[..., 0] > 0)
    vol = ((2 * math.pi) ** (4 - 3 * n) * (math.pi / 2) ** (n - 1) * rs ** (2 * n - 4)
           / (math.factorial(n - 1) * math.factorial(n - 2)))
    np.testing.assert_allclose(w, vol, rtol=1e-15)
    if n == 2:
        assert ps.massless_volume(2, 7.0) == pytest.approx(1 / (8 * math.pi), rel=1e-15)


@pytest.mark.parametrize("n", [3, 4])
def test_rambo_diet_matches_classic_rambo(n):
    rng = np.random.default_rng(10 + n)
    N = 60000
    pd, _ = ps.rambo_diet(1000.0, rng.random((3 * n - 4, N)), n)
    pc, _ = ps.rambo_classic(1000.0, rng.random((4 * n, N)), n)
    for i in range(n):
        for j in range(i + 1, n):
            sd = mdot(pd[:, i] + pd[:, j], pd[:, i] + pd[:, j])
            sc = mdot(pc[:, i] + pc[:, j], pc[:, i] + pc[:, j])
            assert stats.ks_2samp(sd, sc).pvalue > 1e-4
        # single-particle energy spectra too
        assert stats.ks_2samp(pd[:, i, 0], pc[:, i, 0]).pvalue > 1e-4


def test_massive_two_body_weight_is_beta_over_8pi():
    rng = np.random.default_rng(4)
    rs, m = 1000.0, 173.0
    p, w = ps.rambo_diet(rs, rng.random((2, 500)), 2)
    k, wm = ps.massive(p, [m, m], rs)
    beta = math.sqrt(1 - 4 * m * m / rs ** 2)
    np.testing.assert_allclose(w * wm, beta / (8 * math.pi), rtol=1e-14)
    np.testing.assert_allclose(mdot(k, k), np.full((500, 2), m * m), rtol=1e-12)


@pytest.mark.parametrize("n", [3, 4])
def test_massive_on_shell_and_conserving(n):
    rng = np.random.default_rng(20 + n)
    rs = 900.0
    masses = [173.0, 173.0] + [0.0] * (n - 2)
    p, _ = ps.rambo_diet(rs, rng.random((3 * n - 4, 1000)), n)
    k, wm = ps.massive(p, masses, rs)
    np.testing.assert_allclose(mdot(k, k), np.broadcast_to(np.array(masses) ** 2, (1000, n)),
                               atol=1e-11 * rs * rs)
    np.testing.assert_allclose(k.sum(axis=1)[:, 0], rs, rtol=1e-11)
    np.testing.assert_allclose(k.sum(axis=1)[:, 1:], 0, atol=1e-11 * rs)
    assert np.all((wm > 0) & (wm <= 1))


def test_massive_three_body_volume_equals_dalitz_area():
    m, rs = 173.0, 700.0
    s = rs * rs

    def m23_range(m12sq):            # particles 1=t (m), 2=tbar (m), 3=g (0)
        E2 = (m12sq - m * m + m * m) / (2 * math.sqrt(m12sq))
        E3 = (s - m12sq - 0.0) / (2 * math.sqrt(m12sq))
        p2 = math.sqrt(max(E2 * E2 - m * m, 0.0))
        p3 = E3
        return (E2 + E3) ** 2 - (p2 + p3) ** 2, (E2 + E3) ** 2 - (p2 - p3) ** 2

    area, _ = integrate.quad(lambda x: m23_range(x)[1] - m23_range(x)[0], (2 * m) ** 2, s,
                             epsabs=0, epsrel=1e-12)
    volume = area / (128 * math.pi ** 3 * s)
    rng = np.random.default_rng(5)
    N = 400000
    p, w = ps.rambo_diet(rs, rng.random((5, N)), 3)
    _, wm = ps.massive(p, [m, m, 0.0], rs)
    ww = w * wm
    mean, err = ww.mean(), ww.std() / math.sqrt(N)
    assert abs(mean - volume) < 4 * err
    assert err / mean < 2e-3


def test_luminosity_map():
    tau0, S = 4 * 173.0 ** 2 / 13000.0 ** 2, 13000.0 ** 2
    rng = np.random.default_rng(6)
    ua, ub = rng.random(500) * 0.98 + 0.01, rng.random(500) * 0.98 + 0.01
    x1, x2, shat, L = ps.luminosity_map(ua, ub, tau0, S)
    assert np.all(x1 * x2 >= tau0 * (1 - 1e-15)) and np.all(x1 <= 1) and np.all(x2 <= 1)
    np.testing.assert_allclose(shat, x1 * x2 * S, rtol=1e-15)
    h = 1e-6
    d1 = (ps.luminosity_map(ua + h, ub, tau0, S)[0] - ps.luminosity_map(ua - h, ub, tau0, S)[0]) / (2 * h)
    d2 = (ps.luminosity_map(ua, ub + h, tau0, S)[1] - ps.luminosity_map(ua, ub - h, tau0, S)[1]) / (2 * h)
    f = lambda x: x ** -1.1 * (1 - x) ** 5
    np.testing.assert_allclose(L, f(x1) * f(x2) * np.abs(d1 * d2), rtol=1e-7)


def test_cuts():
    k = np.zeros((3, 4, 4))
    # event 0: gluons at pT 40 and 50, far apart; event 1: one soft gluon;
    # event 2: two hard gluons almost collinear
    def g(pt_, y, phi):
        return [pt_ * math.cosh(y), pt_ * math.cos(phi), pt_ * math.sin(phi), pt_ * math.sinh(y)]
    k[0, 2], k[0, 3] = g(40, 0.1, 0.0), g(50, -1.0, 2.0)
    k[1, 2], k[1, 3] = g(20, 0.1, 0.0), g(50, -1.0, 2.0)
    k[2, 2], k[2, 3] = g(40, 0.1, 3.1), g(50, 0.2, -3.1)    # dphi wraps to 0.083
    ok = ps.pass_cuts(k, [2, 3], 30.0, 0.4)
    assert list(ok) == [True, False, False]
    assert ps.delta_r(np.array(g(40, 0.1, 3.1)), np.array(g(50, 0.2, -3.1))) == pytest.approx(
        math.hypot(0.1, 2 * math.pi - 6.2), rel=1e-12)
    assert list(ps.pass_cuts(k, [2, 3], 0.0, 0.0)) == [True, True, True]
