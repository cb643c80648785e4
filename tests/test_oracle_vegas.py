"""Pins for oracle.vegas (Lepage's algorithm; arXiv:2211.14056 Sec. 1 cites it).

* the uniform grid maps y to itself with unit Jacobian;
* bins come from the IEEE product floor(y * 50), clamped;
* a constant integrand leaves the grid where it is;
* a separable integrand of known integral is estimated within 3 sigma and the
  adapted grid approaches the inverse CDF of |f| in each dimension;
* the combination is the inverse-variance mean with its chi^2.
"""
import math

import numpy as np
import pytest

from oracle import vegas


def test_uniform_grid_is_identity():
    rng = np.random.default_rng(0)
    y = rng.random((3, 1000))
    x, jac, bins = vegas.vegas_map(y, vegas.uniform_grid(3))
    np.testing.assert_allclose(x, y, rtol=0, atol=1e-15)
    np.testing.assert_allclose(jac, 1.0, rtol=1e-13)
    np.testing.assert_array_equal(bins, np.floor(y * 50).astype(int))


def test_bin_clamp_and_edges():
    e = vegas.uniform_grid(1)
    y = np.array([[0.0, 0.02, 1.0 - 2.0 ** -53, 1.0]])
    _, _, b = vegas.vegas_map(y, e)
    assert list(b[0]) == [0, 1, 49, 49]


def test_jacobian_matches_numerical_derivative():
    rng = np.random.default_rng(1)
    e = np.sort(np.concatenate([[0.0, 1.0], rng.random(49)]))[None, :]
    y = rng.random((1, 200)) * 0.98 + 0.01
    h = 1e-7
    x, jac, b = vegas.vegas_map(y, e)
    xp, _, bp = vegas.vegas_map(y + h, e)
    same = bp[0] == b[0]
    np.testing.assert_allclose(((xp - x) / h)[0][same], jac[same], rtol=1e-5)


def test_constant_integrand_keeps_grid():
    rng = np.random.default_rng(2)
    e = np.sort(np.concatenate([[0.0, 1.0], rng.random(49)]))
    d = np.full(50, 3.7)
    np.testing.assert_allclose(vegas.refine_dim(e, d), e, rtol=0, atol=4e-16)
    # all-zero histogram: unchanged
    np.testing.assert_array_equal(vegas.refine_dim(e, np.zeros(50)), e)


def test_refine_edge_cases():
    e = np.linspace(0, 1, 51)
    d = np.zeros(50)
    d[10] = 1.0                        # all weight in one bin before smoothing
    new = vegas.refine_dim(e, d)
    assert new[0] == 0 and new[-1] == 1 and np.all(np.diff(new) > 0)
    assert np.all((new[1:-1] >= e[9]) & (new[1:-1] <= e[12]))


def test_separable_integrand_converges():
    # f(x) = prod_j g(x_j), g(x) = 3 x^2 on [0,1]: integral 1, optimal map x = y^(1/3)
    rng = np.random.default_rng(3)
    edges = vegas.uniform_grid(2)
    means, variances = [], []
    for it in range(8):
        y = rng.random((2, 20000))
        x, jac, bins = vegas.vegas_map(y, edges)
        w = np.prod(3 * x ** 2, axis=0) * jac
        sw, sw2, hist = vegas.accumulate(w, bins)
        I, var = vegas.estimate(sw, sw2, y.shape[1])
        means.append(I)
        variances.append(var)
        edges = vegas.refine(edges, hist)
    I, sig, chi2 = vegas.combine(means[2:], variances[2:])
    assert abs(I - 1.0) < 3 * sig
    target = np.linspace(0, 1, 51) ** (1.0 / 3.0)
    err = np.abs(edges - target[None, :])
    # smoothing and damping bias the first bins; the bulk sits on the inverse CDF
    assert np.max(err) < 0.05 and np.mean(err) < 0.01
    assert np.max(err) < 0.25 * np.max(np.abs(np.linspace(0, 1, 51) - target))


def test_estimate_and_combine():
    I, var = vegas.estimate(10.0, 30.0, 4)
    assert I == 2.5 and var == pytest.approx((7.5 - 6.25) / 3)
    m, s, chi2 = vegas.combine([1.0, 3.0], [1.0, 1.0])
    assert m == 2.0 and s == pytest.approx(1 / math.sqrt(2)) and chi2 == pytest.approx(2.0)
    m, s, chi2 = vegas.combine([1.0, 2.0], [1.0, 4.0])
    assert m == pytest.approx((1 + 0.5) / 1.25)
    with pytest.raises(ValueError):
        vegas.combine([1.0], [0.0])


def test_histogram_sums_w_squared_per_bin():
    w = np.array([1.0, 2.0, 3.0])
    bins = np.array([[0, 0, 49], [5, 6, 5]])
    sw, sw2, h = vegas.accumulate(w, bins)
    assert sw == 6 and sw2 == 14
    assert h[0, 0] == 5 and h[0, 49] == 9 and h[1, 5] == 10 and h[1, 6] == 4
