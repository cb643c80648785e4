"""Pins for the oracle's |M|^2 (oracle.feynman, oracle.berends_giele, oracle.processes).

* diagram counts of the enumerator: 3 / 16 / 123 (gg -> t tbar + 0/1/2 g);
* closed forms: gg -> t tbar (Combridge 1979; Ellis-Stirling-Webber Table 7.1),
  u ubar -> t tbar, e+ e- -> mu+ mu- (photon exchange), per event;
* gauge invariance: eps_j -> k_j makes the amplitude vanish (Gamma_t = 0);
* Lorentz invariance under random boosts and rotations;
* Bose symmetry of identical gluons;
* two independent algorithms agree: Feynman diagrams with explicit colour vs
  colour-ordered recursion with the trace-basis colour matrix;
* massless limit: the helicity configurations that must vanish do, and the
  MHV partial amplitudes follow the Parke-Taylor form |<f- j>^3 <f+ j>|^2 / prod|s|;
* |M|^2 scales as g_s^(2 (n_ext - 2)).
* helicity-flip symmetry at Gamma_t = 0: |M_h|^2 = |M_-h|^2 per helicity
  configuration, and the per-helicity values of the two algorithms agree.
* the other subprocesses of p p -> t tbar g g (incoming antiquark, incoming
  gluon with an outgoing quark): massless 2 -> 2 closed forms with the same
  external states (q g -> q g, q qbar -> g g, g g -> q qbar; Ellis-Stirling-
  Webber Table 7.1), crossing keeps the diagram count, gauge and Lorentz
  invariance, and the relations between channels: exchanging the beams, and
  charge conjugation (q~ g -> t t~ g q~ equals q g -> t~ t g q with the top
  and antitop momenta exchanged).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import phase_space as ps
from oracle.berends_giele import QQbarGluons
from oracle.feynman import DiagramSet
from oracle.processes import Process, outgoing_flavours


def mdot(a, b):
    return a[..., 0] * b[..., 0] - np.sum(a[..., 1:] * b[..., 1:], axis=-1)


def points(nfin, N, rs=1500.0, masses=None, seed=0):
    rng = np.random.default_rng(seed)
    masses = masses if masses is not None else [173.0, 173.0] + [0.0] * (nfin - 2)
    p = np.zeros((N, nfin + 2, 4))
    p[:, 0] = [rs / 2, 0, 0, rs / 2]
    p[:, 1] = [rs / 2, 0, 0, -rs / 2]
    pm, _ = ps.rambo_diet(rs, rng.random((3 * nfin - 4, N)), nfin)
    p[:, 2:], _ = ps.massive(pm, masses, rs)
    return p


@pytest.mark.parametrize("name,count", [("gg_ttx", 3), ("gg_ttxg", 16), ("gg_ttxgg", 123),
                                        ("uux_ttx", 1), ("epem_mupmum", 1)])
def test_diagram_counts(name, count):
    assert len(DiagramSet(outgoing_flavours(name)).diagrams) == count


def test_gg_ttx_closed_form():
    mt, rs = 173.0, 1000.0
    p = points(2, 40, rs, seed=1)
    proc = Process("gg_ttx", mt=mt)
    s = rs * rs
    t1, t2, rho = 2 * mdot(p[:, 0], p[:, 2]) / s, 2 * mdot(p[:, 1], p[:, 2]) / s, 4 * mt * mt / s
    ref = proc.gs ** 4 * (1 / (6 * t1 * t2) - 3 / 8) * (t1 ** 2 + t2 ** 2 + rho - rho ** 2 / (4 * t1 * t2))
    np.testing.assert_allclose(proc.me2(p), ref, rtol=1e-13)


def test_uux_ttx_closed_form():
    mt, rs = 173.0, 800.0
    p = points(2, 40, rs, seed=2)
    proc = Process("uux_ttx", mt=mt)
    s = rs * rs
    t1, t2, rho = 2 * mdot(p[:, 0], p[:, 2]) / s, 2 * mdot(p[:, 1], p[:, 2]) / s, 4 * mt * mt / s
    ref = proc.gs ** 4 * (4 / 9) * (t1 ** 2 + t2 ** 2 + rho / 2)
    np.testing.assert_allclose(proc.me2(p), ref, rtol=1e-13)


def test_ee_mumu_closed_form():
    rs = 91.0
    p = points(2, 40, rs, masses=[0.0, 0.0], seed=3)
    proc = Process("epem_mupmum")
    s = rs * rs
    cos = p[:, 2, 3] / p[:, 2, 0]
    np.testing.assert_allclose(proc.me2(p), proc.ee ** 4 * (1 + cos ** 2), rtol=1e-13)


def _gauge_ratio(proc, p, leg):
    ext, q = proc.external(p)
    k = p[:, leg].astype(complex)
    ext2 = list(ext)
    ext2[leg] = np.broadcast_to(k[None], (2,) + k.shape).reshape(ext[leg].shape)
    K = proc.amp.amplitude_terms(ext2, q)
    c = proc.amp.colour_terms()
    M = np.einsum("tc,th->ch", c, K.reshape(K.shape[0], -1))
    single = np.max(np.abs(c)) * np.max(np.abs(K))
    return np.max(np.abs(M)) / single


@pytest.mark.parametrize("name,nfin", [("gg_ttxg", 3), ("gg_ttxgg", 4), ("uux_ttxgg", 4), ("ug_ttxgu", 4),
                                       ("gux_ttxgux", 4)])
def test_gauge_invariance(name, nfin):
    proc = Process(name, wt=0.0)
    p = points(nfin, 6, seed=4)
    for leg, part in enumerate(proc.particles):
        if part == "g":
            assert _gauge_ratio(proc, p, leg) < 1e-12


def _random_lorentz(rng):
    # rotation
    A = rng.normal(size=(3, 3))
    Q, _ = np.linalg.qr(A)
    R = np.eye(4)
    R[1:, 1:] = Q * np.sign(np.linalg.det(Q))
    # boost
    b = rng.normal(size=3)
    b *= rng.uniform(0.1, 0.9) / np.linalg.norm(b)
    g = 1 / math.sqrt(1 - b @ b)
    B = np.eye(4)
    B[0, 0] = g
    B[0, 1:] = B[1:, 0] = g * b
    B[1:, 1:] += (g - 1) * np.outer(b, b) / (b @ b)
    return B @ R


@pytest.mark.parametrize("name,nfin", [("gg_ttxg", 3), ("gg_ttxgg", 4), ("uux_ttxgg", 4), ("ug_ttxgu", 4),
                                       ("uxg_ttxgux", 4)])
def test_lorentz_invariance(name, nfin):
    # Gamma_t = 0: a fixed-width propagator breaks gauge invariance at
    # O(Gamma/m), and with it the frame independence of the physical-
    # polarisation sum, so the exact statement is made at zero width
    rng = np.random.default_rng(5)
    proc = Process(name, wt=0.0)
    p = points(nfin, 6, seed=6)
    L = _random_lorentz(rng)
    pb = np.einsum("mn,ejn->ejm", L, p)
    np.testing.assert_allclose(proc.me2(pb), proc.me2(p), rtol=1e-11)


def test_bose_symmetry():
    proc = Process("gg_ttxgg", wt=1.5)
    p = points(4, 6, seed=7)
    ref = proc.me2(p)
    np.testing.assert_allclose(proc.me2(p[:, [1, 0, 2, 3, 4, 5]]), ref, rtol=1e-12)
    np.testing.assert_allclose(proc.me2(p[:, [0, 1, 2, 3, 5, 4]]), ref, rtol=1e-12)


@pytest.mark.parametrize("name,nfin,wt", [("gg_ttx", 2, 0.0), ("gg_ttxg", 3, 0.0), ("gg_ttxg", 3, 1.5),
                                          ("gg_ttxgg", 4, 1.5)])
def test_recursion_agrees_with_feynman_diagrams(name, nfin, wt):
    proc = Process(name, wt=wt)
    p = points(nfin, 12, seed=8)
    np.testing.assert_allclose(QQbarGluons(proc).me2(p), proc.me2(p), rtol=2e-12)


def test_coupling_power_law():
    p = points(4, 4, seed=9)
    a = Process("gg_ttxgg", wt=1.5, gs=1.0).me2(p)
    b = Process("gg_ttxgg", wt=1.5, gs=1.3).me2(p)
    np.testing.assert_allclose(b / a, 1.3 ** 8, rtol=1e-12)


@pytest.mark.parametrize("name,nfin", [("gg_ttxg", 3), ("gg_ttxgg", 4)])
def test_massless_helicity_selection_and_parke_taylor(name, nfin):
    proc = Process(name, mt=0.0)
    bg = QQbarGluons(proc)
    p = points(nfin, 5, rs=1000.0, masses=[0.0] * nfin, seed=10)
    J = bg.partial_amplitudes(p)                  # [sigma, h0..h_{n-1}, N]
    n = len(proc.particles)
    q = np.where(np.array(proc.incoming)[None, :, None], -p, p)
    s = lambda i, j: np.abs(mdot(q[:, i] + q[:, j], q[:, i] + q[:, j]))
    scale = np.max(np.abs(J))
    ratios = []
    for hel in itertools.product((0, 1), repeat=n):
        lam = [(-1, 1)[h] for h in hel]
        out = [-l if inc else l for l, inc in zip(lam, proc.incoming)]   # crossing flips helicity
        neg = [i for i in range(n) if out[i] < 0]
        pos = [i for i in range(n) if out[i] > 0]
        Jh = J[(slice(None),) + hel]
        alive = out[bg.t] == -out[bg.tb] and len(neg) >= 2 and len(pos) >= 2
        if not alive:
            assert np.max(np.abs(Jh)) < 1e-12 * scale
            continue
        assert np.max(np.abs(Jh)) > 1e-6 * scale
        if len(neg) == 2 or len(pos) == 2:
            few = neg if len(neg) == 2 else pos
            f1 = bg.t if bg.t in few else bg.tb
            f2 = bg.tb if f1 == bg.t else bg.t
            j = [i for i in few if i != f1][0]
            for si, order in enumerate(bg.orders):
                cyc = [bg.t] + [bg.gluons[o] for o in order] + [bg.tb]
                den = np.prod([s(cyc[a], cyc[(a + 1) % len(cyc)]) for a in range(len(cyc))], axis=0)
                pt = s(f1, j) ** 3 * s(f2, j) / den
                ratios.append(np.abs(Jh[si]) ** 2 / pt)
    ratios = np.array(ratios)
    np.testing.assert_allclose(ratios, ratios.flat[0], rtol=1e-10)


def _per_helicity(proc, p):
    """Colour-summed |M_h|^2 for every helicity configuration h, shape
    (2,) * n_ext + (N,), from the Feynman-diagram terms with explicit colour."""
    ext, q = proc.external(p)
    K = proc.amp.amplitude_terms(ext, q)
    c = proc.amp.colour_terms()
    M = np.einsum("tc,th->ch", c, K.reshape(K.shape[0], -1))
    per = np.sum(np.abs(M) ** 2, axis=0)
    return per.reshape((2,) * len(proc.particles) + (p.shape[0],))


@pytest.mark.parametrize("name,nfin,masses", [("gg_ttxg", 3, None), ("gg_ttxgg", 4, None),
                                              ("uux_ttxgg", 4, None), ("epem_mupmum", 2, [0.0, 0.0])])
def test_helicity_flip_symmetry(name, nfin, masses):
    """At Gamma_t = 0 every tree amplitude here is built from real momenta,
    real couplings and helicity states whose flipped counterparts are their
    conjugates up to phases (parity followed by complex conjugation), so the
    colour-summed |M|^2 of each helicity configuration equals that of the
    configuration with every helicity reversed, event by event, also for the
    non-planar 2 -> 3 and 2 -> 4 kinematics.  A phase or sign slip between the
    two helicity states of any external wavefunction breaks it."""
    proc = Process(name, wt=0.0)
    p = points(nfin, 5, masses=masses, seed=8)
    per = _per_helicity(proc, p)
    flip = per[(slice(None, None, -1),) * len(proc.particles)]
    scale = np.max(per.reshape(-1, p.shape[0]), axis=0)
    assert np.max(np.abs(flip - per) / scale) < 1e-12
    if name.startswith("gg"):
        bg = QQbarGluons(proc)
        J = bg.partial_amplitudes(p)
        Jf = J.reshape(J.shape[0], -1, J.shape[-1])
        perbg = np.real(np.einsum("shn,st,thn->hn", np.conj(Jf), bg.C, Jf)).reshape(per.shape)
        np.testing.assert_allclose(perbg, per, rtol=0, atol=1e-12 * scale.max())


def _mandelstam(p):
    s = mdot(p[:, 0] + p[:, 1], p[:, 0] + p[:, 1])
    t = mdot(p[:, 0] - p[:, 2], p[:, 0] - p[:, 2])
    u = mdot(p[:, 0] - p[:, 3], p[:, 0] - p[:, 3])
    return s, t, u


@pytest.mark.parametrize("name", ["ug_ug", "uux_gg", "gg_uux"])
def test_massless_two_to_two_closed_forms(name):
    """Spin- and colour-averaged |M|^2 / g^4 of Ellis-Stirling-Webber Table 7.1
    (massless, t = (p1 - p3)^2, u = (p1 - p4)^2); the process's 1/2! for two
    final gluons is part of the oracle's |M|^2."""
    p = points(2, 40, 700.0, masses=[0.0, 0.0], seed=11)
    proc = Process(name)
    s, t, u = _mandelstam(p)
    if name == "ug_ug":
        ref = -(4 / 9) * (s * s + u * u) / (s * u) + (u * u + s * s) / (t * t)
    elif name == "uux_gg":
        ref = ((32 / 27) * (t * t + u * u) / (t * u) - (8 / 3) * (t * t + u * u) / (s * s)) / 2
    else:
        ref = (1 / 6) * (t * t + u * u) / (t * u) - (3 / 8) * (t * t + u * u) / (s * s)
    np.testing.assert_allclose(proc.me2(p), proc.gs ** 4 * ref, rtol=1e-12)


def test_crossing_keeps_the_diagram_count():
    n = len(DiagramSet(outgoing_flavours("uux_ttxgg")).diagrams)
    for name in ("uxu_ttxgg", "ug_ttxgu", "gu_ttxgu", "uxg_ttxgux", "gux_ttxgux"):
        assert len(DiagramSet(outgoing_flavours(name)).diagrams) == n


@pytest.mark.parametrize("wt", [0.0, 1.5])
def test_beam_exchange_and_charge_conjugation(wt):
    p = points(4, 8, seed=12)
    beams = p[:, [1, 0, 2, 3, 4, 5]]
    tops = p[:, [0, 1, 3, 2, 4, 5]]
    me = lambda name, q: Process(name, wt=wt).me2(q)
    np.testing.assert_allclose(me("uxu_ttxgg", p), me("uux_ttxgg", beams), rtol=1e-12)
    np.testing.assert_allclose(me("gu_ttxgu", p), me("ug_ttxgu", beams), rtol=1e-12)
    np.testing.assert_allclose(me("gux_ttxgux", p), me("uxg_ttxgux", beams), rtol=1e-12)
    np.testing.assert_allclose(me("uxg_ttxgux", p), me("ug_ttxgu", tops), rtol=1e-12)
    np.testing.assert_allclose(me("gux_ttxgux", p), me("gu_ttxgu", tops), rtol=1e-12)
