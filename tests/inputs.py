"""Seeded synthetic inputs shared by the oracle and CUDA sides of the tests.

Holds no arithmetic of the method: only seeds, random (but valid) Vegas grids
and event-index samples drawn with numpy's default generator.
"""
import numpy as np


def random_grid(ndim, nbins=50, seed=0):
    """Strictly increasing edges on [0, 1] with bins of uneven width."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.2, 1.8, size=(ndim, nbins))
    e = np.concatenate([np.zeros((ndim, 1)), np.cumsum(w, axis=1)], axis=1)
    e /= e[:, -1:]
    e[:, -1] = 1.0
    return e


def event_sample(n_total, k, seed=0):
    """k distinct global event indices out of n_total, sorted."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_total, size=k, replace=False)).astype(np.uint64)
