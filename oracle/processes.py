"""Process definitions and the per-event |M|^2 the path returns.

Test infrastructure (see ``oracle/__init__``).

|M|^2 = (1 / A) (1 / S_id) sum_helicities sum_colours |M_h|^2
with A the initial-state spin x colour average (gg: 4*64, q qbar: 4*9,
e+e-: 4) and S_id = k! for k identical final-state particles (MadGraph's
convention; arXiv:2211.14056 is silent on it).  Particle order follows
MadGraph: the two incoming partons, then t, tbar, then final gluons.

Momenta: array [N, n, 4] of physical momenta (incoming ones with positive
energy), components (E, px, py, pz).
"""
import math
import numpy as np

from . import wavefunctions as wf
from .feynman import DiagramSet, Amplitude

ALPHA_EM = 1.0 / 137.035999


# name -> (physical particles, incoming flags, average, identical-particle factor)
PROCESSES = {
    "gg_ttx":     (("g", "g", "t", "t~"), (True, True, False, False), 256, 1),
    "gg_ttxg":    (("g", "g", "t", "t~", "g"), (True, True, False, False, False), 256, 1),
    "gg_ttxgg":   (("g", "g", "t", "t~", "g", "g"), (True, True, False, False, False, False), 256, 2),
    "uux_ttxgg":  (("u", "u~", "t", "t~", "g", "g"), (True, True, False, False, False, False), 36, 2),
    "uux_ttx":    (("u", "u~", "t", "t~"), (True, True, False, False), 36, 1),
    "epem_mupmum": (("e-", "e+", "mu-", "mu+"), (True, True, False, False), 4, 1),
    # the other subprocesses of p p -> t tbar g g (the antiquark or a quark from
    # either beam; other light flavours have the same |M|^2): average over the
    # spins and colours of q g = 2*3 x 2*8 = 96; one final gluon, so S_id = 1
    "uxu_ttxgg":  (("u~", "u", "t", "t~", "g", "g"), (True, True, False, False, False, False), 36, 2),
    "ug_ttxgu":   (("u", "g", "t", "t~", "g", "u"), (True, True, False, False, False, False), 96, 1),
    "gu_ttxgu":   (("g", "u", "t", "t~", "g", "u"), (True, True, False, False, False, False), 96, 1),
    "uxg_ttxgux": (("u~", "g", "t", "t~", "g", "u~"), (True, True, False, False, False, False), 96, 1),
    "gux_ttxgux": (("g", "u~", "t", "t~", "g", "u~"), (True, True, False, False, False, False), 96, 1),
    # massless 2 -> 2 processes with textbook closed forms (pins of the
    # external states the crossed processes use: incoming antiquark, incoming
    # gluon with an outgoing quark)
    "ug_ug":      (("u", "g", "u", "g"), (True, True, False, False), 96, 1),
    "uux_gg":     (("u", "u~", "g", "g"), (True, True, False, False), 36, 2),
    "gg_uux":     (("g", "g", "u", "u~"), (True, True, False, False), 256, 1),
}

_ANTI = {"t": "t~", "t~": "t", "u": "u~", "u~": "u", "g": "g", "a": "a",
         "e-": "e+", "e+": "e-", "mu-": "mu+", "mu+": "mu-"}
_PARTICLE = {"t", "u", "e-", "mu-"}
_ANTIPARTICLE = {"t~", "u~", "e+", "mu+"}


def outgoing_flavours(name):
    parts, incoming, _, _ = PROCESSES[name]
    return tuple(_ANTI[p] if inc else p for p, inc in zip(parts, incoming))


def final_gluons(name):
    parts, incoming, _, _ = PROCESSES[name]
    return [i for i, (p, inc) in enumerate(zip(parts, incoming)) if p == "g" and not inc]


def final_jets(name):
    """Final-state light partons (gluons and light quarks): the cuts apply to
    each of them (for processes whose only light final partons are gluons,
    the same as ``final_gluons``)."""
    parts, incoming, _, _ = PROCESSES[name]
    return [i for i, (p, inc) in enumerate(zip(parts, incoming)) if p in ("g", "u", "u~") and not inc]


class Process:
    """Feynman-diagram |M|^2 of one process at fixed couplings and masses."""

    def __init__(self, name, mt=173.0, wt=0.0, gs=1.2177, ee=None):
        self.name = name
        parts, incoming, avg, sid = PROCESSES[name]
        self.particles, self.incoming = parts, incoming
        self.average = avg * sid
        self.mass = {"t": mt, "t~": mt}
        width = {"t": wt, "t~": wt}
        if ee is None:
            ee = math.sqrt(4 * math.pi * ALPHA_EM)
        self.gs, self.ee = gs, ee
        self.diagrams = DiagramSet(outgoing_flavours(name))
        self.amp = Amplitude(self.diagrams, self.mass, width, {"gs": gs, "e": ee})

    def external(self, p):
        """External wavefunctions (leg i carries helicity axis i) and
        outgoing-convention momenta."""
        N, n, _ = p.shape
        ext, q = [], []
        for i, (part, inc) in enumerate(zip(self.particles, self.incoming)):
            m = self.mass.get(part, 0.0)
            states = []
            for lam in (-1, 1):
                if part in ("g", "a"):
                    e = wf.polarisation(p[:, i], lam)
                    states.append(e if inc else np.conj(e))
                elif part in _PARTICLE:
                    u = wf.u_spinor(p[:, i], m, lam)
                    states.append(u if inc else wf.bar(u))
                else:
                    v = wf.v_spinor(p[:, i], m, lam)
                    states.append(wf.bar(v) if inc else v)
            arr = np.stack(states)                     # [2, N, 4]
            shape = [1] * n + [N, 4]
            shape[i] = 2
            ext.append(arr.reshape(shape))
            q.append(-p[:, i] if inc else p[:, i].copy())
        return ext, q

    def me2(self, p):
        """Spin/colour averaged, helicity and colour summed |M|^2 per event."""
        p = np.asarray(p, dtype=np.float64)
        ext, q = self.external(p)
        return self.amp.summed_squared(ext, q) / self.average

    def me2_batched(self, p, batch=256):
        out = np.empty(p.shape[0])
        for s in range(0, p.shape[0], batch):
            out[s:s + batch] = self.me2(p[s:s + batch])
        return out
