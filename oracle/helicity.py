"""Helicity sampling: the |M|^2 of one helicity configuration and the
sampled estimator of the helicity sum.

Test infrastructure (see ``oracle/__init__``).

|M|^2 = (1/A) sum_h |M_h|^2 (``processes``).  Drawing one configuration of
the gluons and the antitop uniformly from the 2^(n_g + 1), summing the top's
two helicities, and weighting by 2^(n_g + 1) estimates that sum without bias
(the practice of MadEvent and MadFlow of sampling helicities instead of
summing them; arXiv:2211.14056 sums them, so the uniform draw is a reading).
The draw comes from the third Philox stream (``philox.helicity_draws``).

Helicity index h, for a top pair plus gluons: bit g (g = 0 .. n_g - 1, the
process's gluons in their order: the two incoming, then the final ones) set
means helicity +1 of that gluon; bit n_g set means antitop helicity +1; the
top is summed.  For the two-quark-line subprocesses of p p -> t t~ g g (a
reading: the bits follow the slots of the u u~ -> t t~ g g amplitude that
the crossed channels fill, and each bit is the helicity of the physical
particle in that slot): bit 0 the incoming quark of the amplitude's light
line (the u, or for u~ g and g u~, whose amplitude is the charge conjugate,
the incoming u~), bit 1 the other light fermion (the incoming u~, or the
outgoing quark of the q g channels), bit 2 the heavy fermion in the antitop
slot (the antitop, or the top for the charge-conjugate channels, where the
antitop is the summed one), bits 3 and 4 the two gluons (for q g the
incoming gluon first).

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


# the legs of bits 0..4 and the summed heavy fermion, per two-quark-line process
_TWO_LINE_LEGS = {
    "uux_ttxgg":  ([0, 1, 3, 4, 5], 2),
    "uxu_ttxgg":  ([1, 0, 3, 4, 5], 2),
    "ug_ttxgu":   ([0, 5, 3, 1, 4], 2),
    "gu_ttxgu":   ([1, 5, 3, 0, 4], 2),
    "uxg_ttxgux": ([0, 5, 2, 1, 4], 3),
    "gux_ttxgux": ([1, 5, 2, 0, 4], 3),
}


def sampled_legs(proc):
    """(legs of bits 0, 1, ..., the summed leg) of a process."""
    if proc.name in _TWO_LINE_LEGS:
        legs, summed = _TWO_LINE_LEGS[proc.name]
        return list(legs), summed
    parts = list(proc.particles)
    gluons = [i for i, x in enumerate(parts) if x == "g"]
    if len(gluons) + 2 != len(parts) or "t" not in parts or "t~" not in parts:
        raise ValueError("helicity sampling covers a top pair plus gluons and the p p -> t t~ g g channels")
    return gluons + [parts.index("t~")], parts.index("t")


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
    the configuration h with the summed heavy fermion's helicity index `top`."""
    legs, summed = sampled_legs(proc)
    hel = np.asarray(hel, dtype=np.int64)
    n = len(proc.particles)
    idx = np.zeros_like(hel)
    for b, leg in enumerate(legs):
        idx += ((hel >> b) & 1) << (n - 1 - leg)
    return idx + (int(top) << (n - 1 - summed))


def me2_helicity(proc, p, hel, algorithm="feynman", amp=None):
    """Per event e: (1/A) (|M_{h_e, -}|^2 + |M_{h_e, +}|^2), the configuration
    h_e, the summed heavy fermion's two helicities added."""
    per = per_helicity(proc, p, algorithm, amp=amp)
    flat = per.reshape(-1, per.shape[-1])
    e = np.arange(flat.shape[1])
    s = flat[config_index(proc, hel, 0), e] + flat[config_index(proc, hel, 1), e]
    return s / proc.average


def n_configs(proc):
    """2^(number of sampled legs): the configurations the draw chooses from."""
    return 2 ** len(sampled_legs(proc)[0])


def sampled_me2(proc, p, hel, algorithm="feynman"):
    """The estimator n_configs me2_helicity of each event."""
    return n_configs(proc) * me2_helicity(proc, p, hel, algorithm)


def sampled_weights(setup, y, edges, seed, iteration, events):
    """Event weights of a Vegas iteration with sampled helicities: the steps of
    ``integrate.Setup.weights`` with |M|^2 replaced by the estimator at the
    configuration drawn for each event (drawn for every event, used where the
    cuts pass).  Returns (w, bins, hel)."""
    p, wk, bins, cut = setup.kinematics(y, edges)
    bits = len(sampled_legs(setup.proc)[0])
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
