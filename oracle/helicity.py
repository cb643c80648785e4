"""Helicity sampling: the |M|^2 of one helicity configuration and the
sampled estimator of the helicity sum.

Test infrastructure (see ``oracle/__init__``).

|M|^2 = (1/A) sum_h |M_h|^2 (``processes``).  Drawing one configuration of
the gluons and the antitop uniformly from the 2^(n_g + 1), summing the top's
two helicities, and weighting by 2^(n_g + 1) estimates that sum without bias
(the practice of MadEvent and MadFlow of sampling helicities instead of
summing them; arXiv:2211.14056 sums them, so the uniform draw is a reading).
The draw comes from the third Philox stream (``philox.helicity_draws``).

Helicity index h: bit g (g = 0 .. n_g - 1, the process's gluons in their
order: the two incoming, then the final ones) set means helicity +1 of that
gluon; bit n_g set means antitop helicity +1.  Processes: a top pair plus
gluons only.

Adapted draw (a reading: MadEvent's choice of helicities by their weight,
written as a discrete Vegas dimension).  The configuration of an event is
drawn from integer thresholds 0 = T_0 <= T_1 <= ... <= T_H = 2^32 by the 32-bit
word w0 of the helicity stream: h = max{h : T_h <= w0}, with probability
p_h = (T_{h+1} - T_h) / 2^32, and the event weighs f_h / p_h.  Uniform
thresholds T_h = h 2^(32 - n_g - 1) give the uniform draw above.  After an
iteration, with S_h the sum of the squared weights of the events drawn in
configuration h, sqrt(p_h S_h) estimates sqrt(N E[f_h^2]) (each event draws
h with probability p_h, and its weight squared is f_h^2 / p_h^2), the choice
of p that minimises the variance; the refined probabilities mix it with the
uniform ones, p'_h = (1 - a) q_h / sum(q) + a / H with q_h = sqrt(p_h S_h),
so that no configuration is left out (unbiasedness needs p_h > 0 wherever f_h
is not zero), and T'_h = floor(2^32 sum_{k<h} p'_k).  Every sum runs in
configuration order, one addition at a time, so that the device, which
rounds each operation separately, computes the same numbers.
"""
import numpy as np

from . import philox


def _legs(proc):
    parts = list(proc.particles)
    gluons = [i for i, x in enumerate(parts) if x == "g"]
    if len(gluons) + 2 != len(parts) or "t" not in parts or "t~" not in parts:
        raise ValueError("helicity sampling covers a top pair plus gluons")
    return gluons, parts.index("t"), parts.index("t~")


def per_helicity(proc, p, algorithm="feynman", batch=256, amp=None):
    """Colour-summed |M_h|^2 of every helicity configuration, shape
    (2,) * n_ext + (N,) (axis i: particle i's helicity, index 0 = -1, 1 = +1),
    not averaged.  algorithm: "feynman" (every diagram with explicit colour;
    amp: another ``feynman.Amplitude`` of the process, e.g. with its diagrams
    rooted at another leg, else the process's own) or "bg" (colour-ordered
    recursion with the trace-basis colour matrix)."""
    p = np.asarray(p, dtype=np.float64)
    n, N = len(proc.particles), p.shape[0]
    out = np.empty((2,) * n + (N,))
    if algorithm == "bg":
        from .berends_giele import QQbarGluons
        bg = QQbarGluons(proc)
    for s in range(0, N, batch):
        q = p[s:s + batch]
        if algorithm == "bg":
            J = bg.partial_amplitudes(q)                 # [sigma, (2,)*n, N]
            v = np.real(np.einsum("s...,st,t...->...", np.conj(J), bg.C, J))
        else:
            a = proc.amp if amp is None else amp
            ext, k = proc.external(q)
            K = a.amplitude_terms(ext, k)                # [term, (2,)*n, N]
            Kf = K.reshape(K.shape[0], -1, K.shape[-1])
            Y = np.einsum("st,thn->shn", a.colour_matrix(), Kf)
            v = np.real(np.einsum("shn,shn->hn", np.conj(Kf), Y)).reshape((2,) * n + (q.shape[0],))
        out[..., s:s + batch] = v
    return out


def config_index(proc, hel, top):
    """Flat index (particle 0 most significant) into the (2,)*n_ext axes of
    the configuration h (gluons and antitop) with top helicity index `top`."""
    gluons, t, tb = _legs(proc)
    hel = np.asarray(hel, dtype=np.int64)
    n, ng = len(proc.particles), len(gluons)
    idx = np.zeros_like(hel)
    for g, leg in enumerate(gluons):
        idx += ((hel >> g) & 1) << (n - 1 - leg)
    idx += ((hel >> ng) & 1) << (n - 1 - tb)
    return idx + (int(top) << (n - 1 - t))


def me2_helicity(proc, p, hel, algorithm="feynman", amp=None):
    """Per event e: (1/A) (|M_{h_e, t-}|^2 + |M_{h_e, t+}|^2), the configuration
    h_e of the gluons and the antitop, the top's two helicities summed."""
    per = per_helicity(proc, p, algorithm, amp=amp)
    flat = per.reshape(-1, per.shape[-1])
    e = np.arange(flat.shape[1])
    s = flat[config_index(proc, hel, 0), e] + flat[config_index(proc, hel, 1), e]
    return s / proc.average


def n_configs(proc):
    """2^(n_g + 1): the configurations the draw chooses from."""
    return 2 ** (len(_legs(proc)[0]) + 1)


def sampled_me2(proc, p, hel, algorithm="feynman"):
    """The estimator 2^(n_g + 1) me2_helicity of each event."""
    return n_configs(proc) * me2_helicity(proc, p, hel, algorithm)


def sampled_weights(setup, y, edges, seed, iteration, events):
    """Event weights of a Vegas iteration with sampled helicities: the steps of
    ``integrate.Setup.weights`` with |M|^2 replaced by the estimator at the
    configuration drawn for each event (drawn for every event, used where the
    cuts pass).  Returns (w, bins, hel)."""
    p, wk, bins, cut = setup.kinematics(y, edges)
    bits = len(_legs(setup.proc)[0]) + 1
    hel = philox.helicity_draws(seed, iteration, events, bits)
    algorithm = "bg" if setup.bg is not None else "feynman"
    w = np.zeros(y.shape[1])
    if np.any(cut):
        w[cut] = sampled_me2(setup.proc, p[cut], hel[cut], algorithm) * wk[cut]
    return w, bins, hel


# ---------------------------------------------------------------------------
# adapted draw

REFINE_FLOOR = 0.1      # the share a of the uniform probabilities kept in a refined table


def uniform_thresholds(n_configs):
    """T_h = h 2^32 / H (H a power of two)."""
    return np.arange(n_configs + 1, dtype=np.int64) * (2 ** 32 // n_configs)


def thresholds(p):
    """T_0..T_H for probabilities p (summing to 1): T_h = floor(2^32 c_h) with
    c_h = p_0 + ... + p_{h-1} added in order, T_0 = 0, T_H = 2^32."""
    p = np.asarray(p, dtype=np.float64)
    c = np.zeros(p.size + 1)
    for h in range(p.size):
        c[h + 1] = c[h] + p[h]
    T = np.floor(c * 2.0 ** 32).astype(np.int64)
    T[0], T[-1] = 0, 2 ** 32
    return np.maximum.accumulate(T)


def probabilities(T):
    """p_h = (T_{h+1} - T_h) / 2^32, the probabilities the thresholds realise."""
    T = np.asarray(T, dtype=np.int64)
    return np.diff(T).astype(np.float64) * 2.0 ** -32


def draw(words, T):
    """h = max{h : T_h <= w0} for each 32-bit word."""
    return np.searchsorted(np.asarray(T, dtype=np.int64), np.asarray(words, dtype=np.int64), side="right") - 1


def refine(T, S, a=REFINE_FLOOR):
    """Refined thresholds from the current ones and the per-configuration sums
    of squared weights S_h; unchanged if every S_h is zero."""
    p = probabilities(T)
    S = np.asarray(S, dtype=np.float64)
    q = np.sqrt(p * S)
    tot = 0.0
    for h in range(q.size):
        tot = tot + q[h]
    if not tot > 0:
        return np.asarray(T, dtype=np.int64).copy()
    H = q.size
    pn = np.empty(H)
    for h in range(H):
        pn[h] = (1.0 - a) * (q[h] / tot) + a / H
    return thresholds(pn)


def adapted_weights(setup, y, edges, seed, iteration, events, T):
    """Event weights of an iteration whose configurations are drawn with the
    thresholds T: f_h / p_h at the drawn h, with f_h = me2_helicity times the
    weight factor.  Returns (w, bins, hel, S) with S_h the sum of the squared
    weights of the events drawn in configuration h."""
    p, wk, bins, cut = setup.kinematics(y, edges)
    T = np.asarray(T, dtype=np.int64)
    hel = draw(philox.helicity_words(seed, iteration, events), T)
    ph = probabilities(T)
    algorithm = "bg" if setup.bg is not None else "feynman"
    w = np.zeros(y.shape[1])
    if np.any(cut):
        w[cut] = me2_helicity(setup.proc, p[cut], hel[cut], algorithm) / ph[hel[cut]] * wk[cut]
    S = np.zeros(T.size - 1)
    np.add.at(S, hel, w * w)
    return w, bins, hel, S
