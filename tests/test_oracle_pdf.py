"""Pins for the oracle's parton-density interpolation (oracle.pdf) and the
tabulated-density luminosity (oracle.phase_space.pdf_luminosity_map).

* node values are returned exactly (to the ln/exp round trip of the query);
* polynomials of degree <= 2 in ln x and in ln Q^2 are reproduced exactly in
  cells whose neighbours exist (uniform nodes make the central difference
  exact for a quadratic), degree <= 1 in every cell;
* along one ln Q^2 node row the 1-D scheme equals scipy's cubic Hermite
  spline given the same node slopes (a library routine);
* the interpolant is C^1 across cell boundaries and converges at third order;
* queries outside the table are clamped to its edge;
* a table of the synthetic gluon density without Q^2 dependence reproduces
  the closed-form luminosity's event weights to its interpolation error;
* the synthetic set is positive below x = 1 and vanishes at x = 1.
"""
import numpy as np
import pytest

from oracle import integrate as oi, philox as oph, vegas as ov
from oracle.pdf import PDFGrid, node_slopes


def _grid(func, nx=21, nq=11, x_min=1e-4, q2_min=4.0, q2_max=1e6, nflav=1):
    t = np.linspace(np.log(x_min), 0.0, nx)
    s = np.linspace(np.log(q2_min), np.log(q2_max), nq)
    T, S = np.meshgrid(t, s)
    xf = np.stack([func(T, S) for _ in range(nflav)])
    return PDFGrid(x_min, 1.0, q2_min, q2_max, xf), t, s


def test_node_values():
    rng = np.random.default_rng(1)
    vals = rng.uniform(0.1, 2.0, size=(2, 11, 21))
    g, t, s = _grid(lambda T, S: 0 * T)
    g = PDFGrid(1e-4, 1.0, 4.0, 1e6, vals)
    for f in range(2):
        for l in (0, 3, 10):
            for k in (0, 7, 20):
                got = g.xfx(f, np.exp(t[k]), np.exp(s[l]))
                assert got == pytest.approx(vals[f, l, k], rel=1e-12)


def test_quadratic_reproduction():
    poly = lambda T, S: (1.0 + 0.5 * T - 0.07 * T * T) * (2.0 - 0.3 * S + 0.02 * S * S)
    g, t, s = _grid(poly)
    rng = np.random.default_rng(2)
    # interior cells: the query's cell and its neighbours exist in both directions
    tt = rng.uniform(t[1], t[-2], 200)
    ss = rng.uniform(s[1], s[-2], 200)
    np.testing.assert_allclose(g.xfx(0, np.exp(tt), np.exp(ss)), poly(tt, ss), rtol=1e-12)
    lin = lambda T, S: 0.3 + 0.2 * T - 0.1 * S + 0.05 * T * S
    g2, _, _ = _grid(lin)
    tt = rng.uniform(t[0], t[-1], 200)
    ss = rng.uniform(s[0], s[-1], 200)
    np.testing.assert_allclose(g2.xfx(0, np.exp(tt), np.exp(ss)), lin(tt, ss), rtol=1e-12, atol=1e-14)


def test_rows_match_scipy_hermite_spline():
    interp = pytest.importorskip("scipy.interpolate")
    f = lambda T, S: np.exp(0.4 * T) * (1.0 + 0.1 * np.sin(S)) + 0.2 * np.cos(3 * T)
    g, t, s = _grid(f)
    rng = np.random.default_rng(3)
    tt = rng.uniform(t[0], t[-1], 100)
    for l in (0, 4, 10):
        row = g.xf[0, l]
        spl = interp.CubicHermiteSpline(t, row, node_slopes(row, t[1] - t[0]))
        np.testing.assert_allclose(g.xfx(0, np.exp(tt), np.exp(s[l])), spl(tt), rtol=1e-11, atol=1e-13)


def test_c1_continuity_across_a_node():
    f = lambda T, S: np.exp(0.4 * T) * (1.0 + 0.1 * np.sin(S))
    g, t, s = _grid(f)
    q2 = np.exp(0.5 * (s[3] + s[4]))
    for k in (5, 12):
        h = 1e-6
        left = (g.xfx(0, np.exp(t[k] - h), q2) - g.xfx(0, np.exp(t[k] - 2 * h), q2)) / h
        right = (g.xfx(0, np.exp(t[k] + 2 * h), q2) - g.xfx(0, np.exp(t[k] + h), q2)) / h
        assert abs(left - right) < 1e-4 * abs(left)
        jump = abs(g.xfx(0, np.exp(t[k] - 1e-12), q2) - g.xfx(0, np.exp(t[k] + 1e-12), q2))
        assert jump < 1e-10


def test_third_order_convergence():
    f = lambda T, S: np.exp(0.3 * T) * np.sin(0.4 * S) + 2.0
    rng = np.random.default_rng(4)
    errs = []
    for nx, nq in ((21, 11), (41, 21), (81, 41)):
        g, t, s = _grid(f, nx=nx, nq=nq)
        tt = rng.uniform(t[2], t[-3], 400)
        ss = rng.uniform(s[2], s[-3], 400)
        errs.append(np.max(np.abs(g.xfx(0, np.exp(tt), np.exp(ss)) - f(tt, ss))))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order > 2.6), (errs, order)


def test_clamping():
    f = lambda T, S: np.exp(0.4 * T) + 0.1 * S
    g, t, s = _grid(f)
    assert g.xfx(0, 1e-9, np.exp(s[3])) == pytest.approx(g.xfx(0, np.exp(t[0]), np.exp(s[3])), rel=1e-14)
    assert g.xfx(0, np.exp(t[5]), 1.0) == pytest.approx(g.xfx(0, np.exp(t[5]), np.exp(s[0])), rel=1e-14)
    assert g.xfx(0, np.exp(t[5]), 1e9) == pytest.approx(g.xfx(0, np.exp(t[5]), np.exp(s[-1])), rel=1e-14)


def test_pdf_luminosity_with_exact_tables_equals_closed_form():
    """Tables the interpolation reproduces exactly (x f constant in x and Q^2:
    1 for one flavour, 2 for another) and two parton pairs give L = 1 + 4 = 5
    times the map's Jacobian: the event weights with lumi = "pdf" equal those
    of the closed-form density f(x) = N x^-1 (1-x)^0 with N^2 = 5, to rounding."""
    nx = 41
    xf = np.stack([np.ones((6, nx)), 2.0 * np.ones((6, nx))])
    base = dict(process="gg_ttxg", mt=173.0, wt=0.0, gs=1.2177, sqrt_s=13000.0, pt_cut=30.0, dr_cut=0.0)
    st1 = oi.Setup(dict(base, lumi=True, lumi_N=np.sqrt(5.0), lumi_a=-1.0, lumi_b=0.0))
    st2 = oi.Setup(dict(base, lumi="pdf", pdf={"x_min": 1e-5, "x_max": 1.0, "q2_min": 1.0, "q2_max": 1e9, "xf": xf},
                        pairs=[(0, 0), (1, 1)], mu_f=0.5))
    y = oph.uniforms(3, 0, np.arange(400, dtype=np.uint64), st1.ndim)
    e = ov.uniform_grid(st1.ndim)
    _, w1, _, c1 = st1.kinematics(y, e)
    _, w2, _, c2 = st2.kinematics(y, e)
    np.testing.assert_array_equal(c1, c2)
    nz = w1 > 0
    assert nz.sum() > 100
    np.testing.assert_allclose(w2[nz], w1[nz], rtol=1e-13)


def test_pdf_luminosity_tracks_the_synthetic_gluon_density():
    """x f(x) = x^(a+1) (1-x)^b tabulated on 801 nodes (no Q^2 dependence):
    the luminosity agrees with the closed form to the interpolation's error
    where the table resolves the density (x1, x2 < 0.3)."""
    from oracle import phase_space as ps
    a, b, nx = -1.1, 5.0, 801
    t = np.linspace(np.log(1e-4), 0.0, nx)
    row = np.exp(t) ** (a + 1) * (1 - np.exp(t)) ** b
    g = PDFGrid(1e-4, 1.0, 1.0, 1e9, np.broadcast_to(row, (1, 5, nx)).copy())
    rng = np.random.default_rng(5)
    tau0, S = 4 * 173.0 ** 2 / 13000.0 ** 2, 13000.0 ** 2
    ua, ub = rng.random(2000), rng.random(2000)
    x1, x2, _, L1 = ps.luminosity_map(ua, ub, tau0, S, 1.0, a, b)
    _, _, _, L2 = ps.pdf_luminosity_map(ua, ub, tau0, S, g, [(0, 0)], 0.5)
    keep = (x1 < 0.3) & (x2 < 0.3)
    assert keep.sum() > 500
    assert np.max(np.abs(L2[keep] / L1[keep] - 1)) < 1e-6


def test_synthetic_set_shape():
    from paper_2211_14056_gb300 import pdfgrid
    d = pdfgrid.synthetic_set()
    xf = d["xf"]
    assert xf.shape == (9, pdfgrid.NQ, pdfgrid.NX)
    assert np.all(xf[:, :, :-1][[0, 1, 2, 3, 4, 5, 6, 7, 8]][:, 1:, :] > 0)   # cbar, c vanish only at the lowest Q^2
    assert np.all(xf[:, :, -1] == 0)                                           # every density vanishes at x = 1
    assert np.all(xf[[1, 2, 3, 4, 5, 6, 7], :, :-1] > 0)
    assert pdfgrid.index(21) == 4 and pdfgrid.index(-2) == 2 and pdfgrid.index(2) == 6
