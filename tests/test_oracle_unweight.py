"""Pins for the oracle's hit-or-miss unweighting (oracle.unweight) and its
random stream (oracle.philox.unweight_uniforms).

* the stream is Philox with the documented counter (word 3 = 1): checked
  against the generator's raw words, and it is uniform and independent of
  the Vegas uniforms of the same events;
* with w_max >= every weight no event is overweight and each is kept with
  probability w / w_max (binomial counts within 5 sigma);
* unbiasedness: w_max * (sum of kept weights) / n equals the mean weight in
  expectation, for any w_max, overweights included (checked over many
  events against the exact mean and its standard error);
* weights <= 0 are never kept; w_max -> infinity keeps nothing; a tiny w_max
  keeps every positive event with weight w / w_max (so the kept weights
  times w_max reproduce the weights exactly).
"""
import numpy as np
import pytest

from oracle import philox
from oracle.unweight import unweight


def test_stream_counter_layout():
    ev = np.arange(5, dtype=np.uint64) + np.uint64(2 ** 33)
    seed, it = 0x1234_5678_9ABC, 3
    w0, w1, _, _ = philox.philox4x32_10(ev & np.uint64(0xFFFFFFFF), ev >> np.uint64(32), np.zeros_like(ev),
                                        np.ones_like(ev), seed & 0xFFFFFFFF, ((seed >> 32) ^ it) & 0xFFFFFFFF)
    np.testing.assert_array_equal(philox.unweight_uniforms(seed, it, ev), philox.words_to_unit(w0, w1))


def test_stream_uniform_and_independent_of_the_vegas_uniforms():
    ev = np.arange(200_000, dtype=np.uint64)
    r = philox.unweight_uniforms(7, 1, ev)
    y = philox.uniforms(7, 1, ev, 2)
    h, _ = np.histogram(r, bins=100, range=(0, 1))
    chi2 = np.sum((h - 2000.0) ** 2 / 2000.0)
    assert chi2 < 99 + 5 * np.sqrt(2 * 99)
    for j in range(2):
        assert abs(np.corrcoef(r, y[j])[0, 1]) < 5 / np.sqrt(ev.size)
        assert not np.any(r == y[j])


def test_acceptance_probability():
    rng = np.random.default_rng(1)
    n = 400_000
    w = np.repeat([0.1, 0.5, 0.9], n // 4).tolist() + [0.0] * (n - 3 * (n // 4))
    w = np.asarray(w)
    r = philox.unweight_uniforms(3, 0, np.arange(w.size, dtype=np.uint64))
    kept, weight = unweight(w, r, 1.0)
    assert np.all(weight == 1.0) and not np.any(kept[w == 0])
    for p in (0.1, 0.5, 0.9):
        m = w == p
        k = kept[m].sum()
        assert abs(k - p * m.sum()) < 5 * np.sqrt(m.sum() * p * (1 - p))


@pytest.mark.parametrize("w_max", [0.05, 0.4, 3.0])
def test_unbiased_with_and_without_overweights(w_max):
    n = 400_000
    rng = np.random.default_rng(2)
    w = rng.exponential(0.2, n) * (rng.random(n) < 0.7)
    r = philox.unweight_uniforms(5, 2, np.arange(n, dtype=np.uint64))
    kept, weight = unweight(w, r, w_max)
    est = w_max * np.sum(weight[kept]) / n
    # per event the estimator is w_max * kept * weight: variance from its moments
    x = w_max * np.where(kept, weight, 0.0)
    assert abs(est - w.mean()) < 5 * x.std() / np.sqrt(n)
    assert np.all(weight[kept & (w > w_max)] > 1) and np.all(weight[kept & (w <= w_max)] == 1)


def test_limits():
    w = np.array([-1.0, 0.0, 1e-3, 0.2, 5.0])
    r = np.array([0.1, 0.5, 0.3, 0.99, 0.5])
    kept, _ = unweight(w, r, 1e300)
    assert kept.tolist() == [False, False, False, False, False]
    kept, weight = unweight(w, r, 1e-10)
    assert kept.tolist() == [False, False, True, True, True]
    np.testing.assert_allclose(weight[kept] * 1e-10, w[kept], rtol=1e-15)
    with pytest.raises(ValueError):
        unweight(w, r, 0.0)
