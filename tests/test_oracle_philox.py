"""Pins for oracle.philox (Philox4x32-10, Salmon et al. SC'11).

* an independent published implementation (Triton's ``tl.philox``, run by its
  CPU interpreter) on arbitrary counters and keys;
* the 53-bit uniform construction: range, resolution and a chi^2 test.
"""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox


def _triton_philox(seed, c0, c1, c2, c3):
    os.environ["TRITON_INTERPRET"] = "1"
    torch = pytest.importorskip("torch")
    triton = pytest.importorskip("triton")
    import triton.language as tl

    @triton.jit
    def kern(out, seed, c0p, c1p, c2p, c3p, N: tl.constexpr):
        o = tl.arange(0, N)
        a = tl.load(c0p + o)
        b = tl.load(c1p + o)
        c = tl.load(c2p + o)
        d = tl.load(c3p + o)
        r0, r1, r2, r3 = tl.philox(seed, a, b, c, d)
        tl.store(out + o * 4 + 0, r0)
        tl.store(out + o * 4 + 1, r1)
        tl.store(out + o * 4 + 2, r2)
        tl.store(out + o * 4 + 3, r3)

    n = len(c0)
    t = lambda x: torch.tensor(np.asarray(x, dtype=np.uint32).view(np.int32))
    out = torch.zeros(4 * n, dtype=torch.int32)
    kern[(1,)](out, seed, t(c0), t(c1), t(c2), t(c3), N=n)
    return out.numpy().view(np.uint32).reshape(n, 4)


def test_philox_matches_triton_reference():
    rng = np.random.default_rng(7)
    n = 16
    c = rng.integers(0, 2 ** 32, size=(4, n), dtype=np.uint64)
    c[:, 0] = 0
    c[:, 1] = 0xFFFFFFFF
    for seed in (0, 1, 0x123456789ABCDEF, 2 ** 63 + 12345):
        ref = _triton_philox(seed, *c)
        got = philox.philox4x32_10(*c, seed & 0xFFFFFFFF, seed >> 32)
        got = np.stack([np.asarray(g, dtype=np.uint64) for g in got], axis=1).astype(np.uint32)
        np.testing.assert_array_equal(got, ref)


def test_stream_layout_uses_key_and_counter_as_documented():
    ev = np.array([0, 5, 2 ** 33 + 7], dtype=np.uint64)
    y = philox.uniforms(seed=(3 << 32) | 11, iteration=2, events=ev, ndim=3)
    k0, k1 = 11, 3 ^ 2
    for j in range(2):
        w = philox.philox4x32_10(ev & np.uint64(0xFFFFFFFF), ev >> np.uint64(32),
                                 np.full(3, j, dtype=np.uint64), np.zeros(3, dtype=np.uint64), k0, k1)
        np.testing.assert_array_equal(y[2 * j], philox.words_to_unit(w[0], w[1]))
        if 2 * j + 1 < 3:
            np.testing.assert_array_equal(y[2 * j + 1], philox.words_to_unit(w[2], w[3]))


def test_unit_construction_range_and_resolution():
    assert philox.words_to_unit(0, 0) == 0.0
    top = philox.words_to_unit(0xFFFFFFFF, 0xFFFFFFFF)
    assert top < 1.0 and top == 1.0 - 2.0 ** -53
    assert philox.words_to_unit(0, 1 << 11) == 2.0 ** -53


def test_uniformity_chi2():
    y = philox.uniforms(1, 0, np.arange(200_000, dtype=np.uint64), 2).ravel()
    counts = np.bincount(np.floor(y * 1000).astype(int), minlength=1000)
    chi2, p = stats.chisquare(counts)
    assert p > 1e-4
    # two dims of one event are not correlated
    y2 = philox.uniforms(1, 0, np.arange(100_000, dtype=np.uint64), 2)
    assert abs(np.corrcoef(y2)[0, 1]) < 0.02
