"""Pins for oracle.helicity (one sampled helicity configuration per event) and
the third Philox stream that draws it.

* completeness: summed over the 2^(n_g + 1) configurations, me2_helicity is
  the helicity-summed |M|^2 of ``processes`` (two algorithms);
* Bose symmetry: exchanging two identical gluons' momenta together with their
  helicity bits leaves a configuration's value unchanged; exchanging the
  momenta alone does not (this places bits 0, 1 on the incoming gluons and
  bits 2, 3 on the final ones);
* charge conjugation: top summed with the antitop's bit b equals, with the top
  and antitop momenta exchanged, the antitop summed with the top's helicity b
  (this places bit n_g on the antitop, not on the top);
* the draw: counter layout of the stream, values in [0, 2^bits), uniform
  (chi^2), independent of the Vegas and the unweighting streams;
* unbiasedness: the estimator's mean over draws is |M|^2 (within 5 sigma),
  and the sampled weights of an iteration integrate to the summed ones;
* the adapted draw: uniform thresholds reproduce the uniform draw exactly;
  the draw's frequencies follow the thresholds' probabilities (chi^2); with
  an adapted table the estimator stays unbiased; the refinement's fixed
  point is the closed-form optimum mixed with the uniform floor, it lowers
  the exact per-event variance on real configurations, keeps every
  probability at or above the floor, and leaves the table alone without data.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import helicity as oh, integrate as oi, philox
from oracle.processes import Process
from tests.test_oracle_amplitudes import points

CASES = [("gg_ttx", 2), ("gg_ttxg", 3), ("gg_ttxgg", 4)]


@pytest.mark.parametrize("name,nfin", CASES)
def test_configurations_sum_to_the_helicity_sum(name, nfin):
    proc = Process(name, wt=1.5)
    nc = oh.n_configs(proc)
    for alg, N in (("feynman", 3), ("bg", 40)):
        p = points(nfin, N, seed=11)
        # every configuration of every event in one call
        v = oh.me2_helicity(proc, np.repeat(p, nc, axis=0), np.tile(np.arange(nc), N), alg)
        tot = v.reshape(N, nc).sum(axis=1)
        assert np.max(np.abs(tot / proc.me2(p) - 1)) < 1e-12
    # the two algorithms agree configuration by configuration
    p = points(nfin, 3, seed=12)
    h = np.arange(3) * 5 % oh.n_configs(proc)
    a, b = oh.me2_helicity(proc, p, h, "feynman"), oh.me2_helicity(proc, p, h, "bg")
    assert np.max(np.abs(a / b - 1)) < 1e-11


def _swap_bits(h, i, j):
    bi, bj = (h >> i) & 1, (h >> j) & 1
    return h & ~((1 << i) | (1 << j)) | (bi << j) | (bj << i)


@pytest.mark.parametrize("name,nfin,legs,bits", [("gg_ttxg", 3, (0, 1), (0, 1)),
                                                  ("gg_ttxgg", 4, (0, 1), (0, 1)),
                                                  ("gg_ttxgg", 4, (4, 5), (2, 3))])
def test_bose_symmetry_places_the_gluon_bits(name, nfin, legs, bits):
    proc = Process(name, wt=1.5)
    N = 24
    p = points(nfin, N, seed=13)
    ps_ = p.copy()
    ps_[:, [legs[0], legs[1]]] = p[:, [legs[1], legs[0]]]
    h = np.arange(N) % oh.n_configs(proc)
    ref = oh.me2_helicity(proc, p, h, "bg")
    got = oh.me2_helicity(proc, ps_, _swap_bits(h, *bits), "bg")
    assert np.max(np.abs(got / ref - 1)) < 1e-10
    # without the bit exchange the configurations with different bits move
    differ = ((h >> bits[0]) & 1) != ((h >> bits[1]) & 1)
    wrong = oh.me2_helicity(proc, ps_, h, "bg")
    assert np.median(np.abs(wrong[differ] / ref[differ] - 1)) > 1e-3


@pytest.mark.parametrize("name,nfin", CASES)
def test_charge_conjugation_places_the_antitop_bit(name, nfin):
    proc = Process(name, wt=1.5)
    N = 16
    p = points(nfin, N, seed=14)
    n = len(proc.particles)
    t, tb = proc.particles.index("t"), proc.particles.index("t~")
    pc = p.copy()
    pc[:, [t, tb]] = p[:, [tb, t]]
    per = oh.per_helicity(proc, pc, "bg")              # (2,)*n + (N,)
    ng = nfin
    h = np.arange(N) * 3 % oh.n_configs(proc)
    got = oh.me2_helicity(proc, p, h, "bg")
    for e in range(N):
        idx = [0] * n
        gl = [i for i, x in enumerate(proc.particles) if x == "g"]
        for g, leg in enumerate(gl):
            idx[leg] = (h[e] >> g) & 1
        idx[t] = (h[e] >> ng) & 1                      # the top takes the antitop's helicity
        s = 0.0
        for a in (0, 1):
            idx[tb] = a
            s += per[tuple(idx) + (e,)]
        assert abs(got[e] * proc.average / s - 1) < 1e-10
    # summing the antitop instead, at the unswapped momenta, would not agree
    # (except for 2 -> 2, whose planar events make the two sums equal)
    if nfin >= 3:
        per0 = oh.per_helicity(proc, p, "bg")
        rel = []
        for e in range(N):
            idx = [0] * n
            for g, leg in enumerate([i for i, x in enumerate(proc.particles) if x == "g"]):
                idx[leg] = (h[e] >> g) & 1
            idx[t] = (h[e] >> ng) & 1
            wrong = sum(per0[tuple(idx[:tb]) + (a,) + tuple(idx[tb + 1:]) + (e,)] for a in (0, 1))
            rel.append(abs(wrong / (got[e] * proc.average) - 1))
        assert np.median(rel) > 1e-4


def test_draw_stream_layout_and_range():
    ev = np.array([0, 9, 2 ** 32 + 3, 2 ** 40 + 1], dtype=np.uint64)
    seed, it = (5 << 32) | 17, 3
    for bits in (3, 4, 5):
        h = philox.helicity_draws(seed, it, ev, bits)
        w = philox.philox4x32_10(ev & np.uint64(0xFFFFFFFF), ev >> np.uint64(32), np.ones(4, dtype=np.uint64),
                                 np.ones(4, dtype=np.uint64), 17, 5 ^ 3)
        np.testing.assert_array_equal(h, (np.asarray(w[0], dtype=np.uint64) >> np.uint64(32 - bits)).astype(np.int64))
        assert h.min() >= 0 and h.max() < 2 ** bits


def test_draws_are_uniform_and_independent():
    n = 320_000
    ev = np.arange(n, dtype=np.uint64)
    h = philox.helicity_draws(7, 2, ev, 5)
    counts = np.bincount(h, minlength=32)
    assert stats.chisquare(counts).pvalue > 1e-4
    # against the unweighting stream and the first Vegas dimension
    r = philox.unweight_uniforms(7, 2, ev)
    y0 = philox.uniforms(7, 2, ev[:100_000], 1)[0]
    assert abs(np.corrcoef(h, r)[0, 1]) < 0.01
    assert abs(np.corrcoef(h[:100_000], y0)[0, 1]) < 0.02
    # another iteration draws other configurations
    assert np.mean(philox.helicity_draws(7, 3, ev[:10000], 5) == h[:10000]) < 0.05


def test_estimator_is_unbiased():
    proc = Process("gg_ttxg", wt=1.5)
    p = points(3, 1, seed=15)
    per = oh.per_helicity(proc, p, "bg").reshape(-1)
    n = 40_000
    h = philox.helicity_draws(3, 0, np.arange(n, dtype=np.uint64), 4)
    v = oh.n_configs(proc) * (per[oh.config_index(proc, h, 0)] + per[oh.config_index(proc, h, 1)]) / proc.average
    me2 = proc.me2(p)[0]
    assert abs(v.mean() - me2) < 5 * v.std() / np.sqrt(n)
    assert v.std() > 0.1 * me2                      # the configurations do differ


def test_sampled_weights_integrate_to_the_summed_ones():
    cfg = dict(process="gg_ttxg", sqrt_s=1000.0, mt=173.0, wt=1.5, pt_cut=20.0, dr_cut=0.4, lumi=False)
    st = oi.Setup(cfg, amplitude="bg")
    n = 6000
    ev = np.arange(n, dtype=np.uint64)
    edges = np.tile(np.linspace(0, 1, 11), (st.ndim, 1))
    y = philox.uniforms(21, 1, ev, st.ndim)
    w_sum, _ = st.weights(y, edges)
    w_s, _, hel = oh.sampled_weights(st, y, edges, 21, 1, ev)
    assert np.all(w_s[w_sum == 0] == 0) and np.all(w_s[w_sum > 0] > 0)
    np.testing.assert_array_equal(hel, philox.helicity_draws(21, 1, ev, 4))
    d = w_s - w_sum                                  # zero mean: E_h[w_s | y] = w_sum
    assert abs(d.mean()) < 5 * d.std() / np.sqrt(n)
    assert np.mean(np.abs(d[w_sum > 0]) > 1e-3 * w_sum[w_sum > 0]) > 0.9   # the draw does move the weights


def test_uniform_thresholds_reproduce_the_uniform_draw():
    ev = np.arange(50_000, dtype=np.uint64)
    for bits in (3, 4, 5):
        T = oh.uniform_thresholds(2 ** bits)
        np.testing.assert_array_equal(oh.draw(philox.helicity_words(9, 4, ev), T), philox.helicity_draws(9, 4, ev, bits))
        assert np.all(oh.probabilities(T) == 2.0 ** -bits)


def test_draw_follows_the_thresholds():
    rng = np.random.default_rng(5)
    p = rng.uniform(0.2, 3.0, 32)
    p /= p.sum()
    T = oh.thresholds(p)
    assert T[0] == 0 and T[-1] == 2 ** 32 and np.all(np.diff(T) > 0)
    assert np.max(np.abs(oh.probabilities(T) - p)) < 2.0 ** -31
    n = 400_000
    h = oh.draw(philox.helicity_words(2, 0, np.arange(n, dtype=np.uint64)), T)
    counts = np.bincount(h, minlength=32)
    assert stats.chisquare(counts, n * oh.probabilities(T)).pvalue > 1e-4


def test_adapted_estimator_is_unbiased():
    proc = Process("gg_ttxg", wt=1.5)
    p = points(3, 1, seed=16)
    per = oh.per_helicity(proc, p, "bg").reshape(-1)
    f = np.array([per[oh.config_index(proc, [h], 0)[0]] + per[oh.config_index(proc, [h], 1)[0]]
                  for h in range(16)]) / proc.average
    T = oh.refine(oh.uniform_thresholds(16), f ** 2 * 16)      # a table adapted to this event
    n = 40_000
    h = oh.draw(philox.helicity_words(4, 0, np.arange(n, dtype=np.uint64)), T)
    v = f[h] / oh.probabilities(T)[h]
    me2 = proc.me2(p)[0]
    assert abs(v.mean() - me2) < 5 * v.std() / np.sqrt(n)
    # adapted to the event itself, the estimator's spread is far below the uniform one's
    vu = 16 * f[philox.helicity_draws(4, 0, np.arange(n, dtype=np.uint64), 4)]
    assert v.std() < 0.5 * vu.std()


def test_refinement_fixed_point_floor_and_no_data():
    rng = np.random.default_rng(7)
    f = rng.uniform(0.0, 1.0, 32) ** 3
    T0 = oh.uniform_thresholds(32)
    p0 = oh.probabilities(T0)
    # expected S for N events: N E[f_h^2 / p_h^2 ; h drawn] = N f_h^2 / p_h
    T1 = oh.refine(T0, 1000.0 * f ** 2 / p0)
    a = oh.REFINE_FLOOR
    want = (1 - a) * f / f.sum() + a / 32
    assert np.max(np.abs(oh.probabilities(T1) - want)) < 2.0 ** -31
    assert np.all(oh.probabilities(T1) >= a / 32 - 2.0 ** -32)
    # the same expectation under the refined table is its own fixed point
    T2 = oh.refine(T1, 1000.0 * f ** 2 / oh.probabilities(T1))
    assert np.max(np.abs(oh.probabilities(T2) - want)) < 2.0 ** -30
    np.testing.assert_array_equal(oh.refine(T1, np.zeros(32)), T1)
    # a configuration never drawn keeps the floor
    S = 1000.0 * f ** 2 / p0
    S[3] = 0.0
    assert abs(oh.probabilities(oh.refine(T0, S))[3] - a / 32) < 2.0 ** -31


def test_refinement_lowers_the_exact_variance():
    """Per-configuration values of 200 gg -> t tbar g events: the exact
    variance of the estimator, sum_h f_h^2 / p_h - (sum_h f_h)^2 averaged
    over the events, drops once the table is refined on the expected sums."""
    proc = Process("gg_ttxg", wt=1.5)
    p = points(3, 200, seed=17)
    f = np.stack([oh.me2_helicity(proc, p, np.full(200, h), "bg") for h in range(16)], axis=1)   # [N, 16]
    T0 = oh.uniform_thresholds(16)

    def var(T):
        ph = oh.probabilities(T)
        return np.mean(np.sum(f ** 2 / ph, axis=1) - f.sum(axis=1) ** 2)

    T1 = oh.refine(T0, np.sum(f ** 2, axis=0) / oh.probabilities(T0))
    print(f"exact variance ratio refined / uniform: {var(T1) / var(T0):.3f}")
    assert var(T1) < var(T0)


def test_adapted_weights_with_uniform_thresholds_equal_the_sampled_weights():
    cfg = dict(process="gg_ttxg", sqrt_s=1000.0, mt=173.0, wt=1.5, pt_cut=20.0, dr_cut=0.4, lumi=False)
    st = oi.Setup(cfg, amplitude="bg")
    n = 600
    ev = np.arange(n, dtype=np.uint64)
    edges = np.tile(np.linspace(0, 1, 11), (st.ndim, 1))
    y = philox.uniforms(22, 1, ev, st.ndim)
    w_s, _, hel_s = oh.sampled_weights(st, y, edges, 22, 1, ev)
    w_a, _, hel_a, S = oh.adapted_weights(st, y, edges, 22, 1, ev, oh.uniform_thresholds(16))
    np.testing.assert_array_equal(hel_a, hel_s)
    np.testing.assert_allclose(w_a, w_s, rtol=1e-15)
    assert abs(S.sum() / np.sum(w_a ** 2) - 1) < 1e-13


# ---------------------------------------------------------------------------
# the two-quark-line subprocesses of p p -> t t~ g g

TWO_LINE = ["uux_ttxgg", "uxu_ttxgg", "ug_ttxgu", "gu_ttxgu", "uxg_ttxgux", "gux_ttxgux"]


def _two_line_points(N, seed):
    return points(4, N, masses=[173.0, 173.0, 0.0, 0.0], seed=seed)


@pytest.mark.parametrize("name", TWO_LINE)
def test_two_line_configurations_sum_and_chirality(name):
    """The 32 configurations sum to the helicity-summed |M|^2, and the massless
    light line conserves chirality: an incoming quark and antiquark that
    annihilate have opposite helicities (u u~, u~ u), a quark or antiquark
    that passes through keeps its helicity (q g -> ... q), so half of the
    configurations vanish exactly: bits 0 and 1 are the light line's two
    fermions."""
    proc = Process(name, wt=1.5)
    assert oh.n_configs(proc) == 32
    N = 2
    p = _two_line_points(N, seed=18)
    v = oh.me2_helicity(proc, np.repeat(p, 32, axis=0), np.tile(np.arange(32), N)).reshape(N, 32)
    assert np.max(np.abs(v.sum(axis=1) / proc.me2(p) - 1)) < 1e-12
    h = np.arange(32)
    annihilate = name in ("uux_ttxgg", "uxu_ttxgg")
    zero = ((h & 1) == ((h >> 1) & 1)) if annihilate else ((h & 1) != ((h >> 1) & 1))
    assert np.all(v[:, zero] <= 1e-25 * v.sum(axis=1, keepdims=True))
    assert np.all(v[:, ~zero].sum(axis=1) > 0)


@pytest.mark.parametrize("a,b,swap", [("uxu_ttxgg", "uux_ttxgg", (0, 1)), ("gu_ttxgu", "ug_ttxgu", (0, 1)),
                                      ("gux_ttxgux", "uxg_ttxgux", (0, 1)), ("uxg_ttxgux", "ug_ttxgu", (2, 3)),
                                      ("gux_ttxgux", "gu_ttxgu", (2, 3))])
def test_two_line_configurations_related_by_beams_and_charge_conjugation(a, b, swap):
    """Per configuration, with the same bits: exchanging the beams relates the
    channels whose quark comes from the other beam; exchanging the top and
    antitop momenta relates a channel to its charge conjugate (the summed and
    the sampled heavy fermion trade places, as the bits say)."""
    pa, pb = Process(a, wt=1.5), Process(b, wt=1.5)
    N = 4
    p = _two_line_points(N, seed=19)
    q = p.copy()
    q[:, [swap[0], swap[1]]] = p[:, [swap[1], swap[0]]]
    h = (np.arange(N) * 9 + 5) % 32
    va, vb = oh.me2_helicity(pa, p, h), oh.me2_helicity(pb, q, h)
    scale = np.maximum(va, vb) + 1e-30
    assert np.max(np.abs(va - vb) / scale) < 1e-10
