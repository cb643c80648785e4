"""Pins for oracle.integrate: the assembled event weight and Vegas iterations.

* gg -> t tbar at sqrt(s) = 1 TeV: the Vegas estimate agrees with the closed
  form sigma = (pi alpha_s^2 / 3s)[(1 + rho + rho^2/16) ln((1+beta)/(1-beta))
  - beta (7/4 + 31 rho/16)] (Combridge 1979) within 3 sigma, and that closed
  form equals Gauss-Legendre quadrature of the differential closed form;
* e+ e- -> mu+ mu- at sqrt(s) = 100 GeV: the estimate agrees with
  4 pi alpha^2 / (3 s) within 3 sigma;
* the hadronic chain (luminosity map, flux, Vegas Jacobian, massive two-body
  phase space) integrates a constant |M|^2 to the 2-D quadrature of
  f(x1) f(x2) beta(s_hat) / (16 pi s_hat);
* iterations are independent of how events are batched (counter-based RNG);
* sums: Kahan and naive summation agree to 1e-13 for these weights.
"""
import math

import numpy as np
import pytest
from scipy import integrate as sint

from oracle import integrate, phase_space as ps, vegas


def sigma_gg_ttx(rs, mt, gs):
    s = rs * rs
    rho = 4 * mt * mt / s
    beta = math.sqrt(1 - rho)
    als = gs * gs / (4 * math.pi)
    return (math.pi * als ** 2 / (3 * s) * ((1 + rho + rho ** 2 / 16) * math.log((1 + beta) / (1 - beta))
                                            - beta * (7 / 4 + 31 * rho / 16))) * ps.GEV2_TO_PB


def test_closed_form_sigma_equals_quadrature_of_dsigma():
    rs, mt, gs = 1000.0, 173.0, 1.2177
    s = rs * rs
    rho = 4 * mt * mt / s
    beta = math.sqrt(1 - rho)

    def dsig(c):           # d sigma / d cos(theta) from the per-event closed form
        t1 = (1 - beta * c) / 2
        t2 = (1 + beta * c) / 2
        me = gs ** 4 * (1 / (6 * t1 * t2) - 3 / 8) * (t1 ** 2 + t2 ** 2 + rho - rho ** 2 / (4 * t1 * t2))
        return me * beta / (32 * math.pi * s) * ps.GEV2_TO_PB
    x, w = np.polynomial.legendre.leggauss(200)
    assert np.sum(w * dsig(x)) == pytest.approx(sigma_gg_ttx(rs, mt, gs), rel=1e-13)


def test_gg_ttx_vegas_matches_closed_form():
    cfg = dict(process="gg_ttx", mt=173.0, wt=0.0, gs=1.2177, sqrt_s=1000.0, lumi=False)
    st = integrate.Setup(cfg)
    res, edges, (I, sig, chi2) = integrate.integrate(st, seed=1, iterations=4, nev=16384)
    ref = sigma_gg_ttx(1000.0, 173.0, 1.2177)
    assert abs(I - ref) < 3 * sig
    assert sig / I < 5e-4


def test_ee_mumu_vegas_matches_closed_form():
    """e+ e- -> mu+ mu- (photon exchange, massless): sigma = 4 pi alpha^2 / (3 s)
    (Peskin-Schroeder Eq. 5.13); the massless two-body phase space (the
    rescaling is the identity) and the flux enter unchanged."""
    cfg = dict(process="epem_mupmum", sqrt_s=100.0, lumi=False)
    st = integrate.Setup(cfg)
    res, edges, (I, sig, chi2) = integrate.integrate(st, seed=2, iterations=4, nev=20000)
    alpha = 1.0 / 137.035999
    ref = 4 * math.pi * alpha ** 2 / (3 * 100.0 ** 2) * ps.GEV2_TO_PB
    assert abs(I - ref) < 3 * sig
    assert sig / I < 2e-4


def test_hadronic_chain_with_constant_matrix_element():
    cfg = dict(process="gg_ttx", mt=173.0, wt=0.0, gs=1.2177, sqrt_s=13000.0, lumi=True)
    st = integrate.Setup(cfg)
    st.me2 = lambda p: np.ones(p.shape[0])
    res, edges, (I, sig, chi2) = integrate.integrate(st, seed=5, iterations=4, nev=20000)
    S = 13000.0 ** 2
    tau0 = 4 * 173.0 ** 2 / S
    f = lambda x: x ** -1.1 * (1 - x) ** 5

    def integrand(x2, x1):
        sh = x1 * x2 * S
        beta = math.sqrt(max(1 - 4 * 173.0 ** 2 / sh, 0.0))
        return f(x1) * f(x2) * beta / (8 * math.pi) / (2 * sh) * ps.GEV2_TO_PB
    ref, _ = sint.dblquad(integrand, tau0, 1.0, lambda x1: tau0 / x1, lambda x1: 1.0, epsrel=1e-9)
    assert abs(I - ref) < 3 * sig


def test_batching_does_not_change_weights():
    cfg = dict(process="gg_ttxg", mt=173.0, wt=0.0, gs=1.2177, sqrt_s=13000.0, lumi=True,
               pt_cut=30.0, dr_cut=0.0)
    st = integrate.Setup(cfg, amplitude="bg")
    edges = vegas.uniform_grid(st.ndim)
    full = integrate.iteration(st, 2, 3, 64, edges)
    part = integrate.iteration(st, 2, 3, 64, edges, events=np.arange(32, 64))
    np.testing.assert_array_equal(full["w"][32:], part["w"])
    np.testing.assert_array_equal(full["bins"][:, 32:], part["bins"])


def test_kahan_and_naive_sums_agree():
    cfg = dict(process="gg_ttxg", mt=173.0, wt=0.0, gs=1.2177, sqrt_s=13000.0, lumi=True,
               pt_cut=30.0, dr_cut=0.0)
    st = integrate.Setup(cfg, amplitude="bg")
    r = integrate.iteration(st, 2, 0, 4096, vegas.uniform_grid(st.ndim))
    w = r["w"]
    s, c = 0.0, 0.0
    for x in w:
        y = x - c
        t = s + y
        c = (t - s) - y
        s = t
    assert abs(s - r["sum_w"]) <= 1e-13 * abs(s)
