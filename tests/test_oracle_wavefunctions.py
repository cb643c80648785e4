"""Pins for oracle.wavefunctions: Dirac equation, completeness, transversality,
including momenta exactly along -z, +z and at rest."""
import numpy as np
import pytest

from oracle import wavefunctions as wf


def _momenta(m, N=50, seed=0):
    rng = np.random.default_rng(seed)
    p3 = rng.normal(size=(N, 3)) * 300
    p3[0] = [0, 0, -250.0]        # exactly along -z
    p3[1] = [0, 0, 250.0]         # exactly along +z
    if m > 0:
        p3[2] = [0, 0, 0]         # at rest
    E = np.sqrt(m * m + np.sum(p3 ** 2, axis=1))
    return np.concatenate([E[:, None], p3], axis=1)


@pytest.mark.parametrize("m", [0.0, 173.0])
def test_dirac_equation_and_completeness(m):
    p = _momenta(m)
    ps = wf.slash(p)
    one = np.eye(4)
    su = np.zeros((p.shape[0], 4, 4), dtype=complex)
    sv = np.zeros_like(su)
    for lam in (-1, 1):
        u = wf.u_spinor(p, m, lam)
        v = wf.v_spinor(p, m, lam)
        np.testing.assert_allclose(np.einsum("nab,nb->na", ps - m * one, u), 0, atol=1e-10 * 300)
        np.testing.assert_allclose(np.einsum("nab,nb->na", ps + m * one, v), 0, atol=1e-10 * 300)
        np.testing.assert_allclose(np.einsum("na,nab->nb", wf.bar(u), ps - m * one), 0, atol=1e-10 * 300)
        su += np.einsum("na,nb->nab", u, wf.bar(u))
        sv += np.einsum("na,nb->nab", v, wf.bar(v))
        # normalisation ubar u = 2m, vbar v = -2m
        np.testing.assert_allclose(np.einsum("na,na->n", wf.bar(u), u), 2 * m, atol=1e-9 * 300)
        np.testing.assert_allclose(np.einsum("na,na->n", wf.bar(v), v), -2 * m, atol=1e-9 * 300)
    np.testing.assert_allclose(su, ps + m * one, atol=1e-10 * 300)
    np.testing.assert_allclose(sv, ps - m * one, atol=1e-10 * 300)


def test_helicity_eigenstates():
    p = _momenta(173.0)
    pa = np.linalg.norm(p[:, 1:], axis=1)
    moving = pa > 0
    # helicity operator Sigma.p/|p| on the right-handed block
    for lam in (-1, 1):
        u = wf.u_spinor(p, 173.0, lam)
        uR = u[:, 2:]
        sp = np.einsum("nk,kab->nab", p[:, 1:] / np.where(moving, pa, 1)[:, None], wf.SIGMA)
        np.testing.assert_allclose(np.einsum("nab,nb->na", sp, uR)[moving], lam * uR[moving], atol=1e-10 * 30)


def test_gamma_algebra():
    g = wf.GAMMA
    for a in range(4):
        for b in range(4):
            np.testing.assert_allclose(g[a] @ g[b] + g[b] @ g[a], 2 * wf.METRIC[a, b] * np.eye(4), atol=1e-15)


def test_polarisation_vectors():
    k = _momenta(0.0)
    for lam in (-1, 1):
        e = wf.polarisation(k, lam)
        np.testing.assert_allclose(wf.mdot(e, k), 0, atol=1e-12 * 300)
        np.testing.assert_allclose(wf.mdot(e, np.conj(e)), -1, atol=1e-14)
        assert np.all(e[:, 0] == 0)
    ep, em = wf.polarisation(k, 1), wf.polarisation(k, -1)
    np.testing.assert_allclose(wf.mdot(ep, np.conj(em)), 0, atol=1e-14)
    # completeness: sum_l e^i e^j* = delta^ij - khat^i khat^j
    kh = k[:, 1:] / np.linalg.norm(k[:, 1:], axis=1)[:, None]
    s = np.einsum("ni,nj->nij", ep[:, 1:], np.conj(ep[:, 1:])) + np.einsum("ni,nj->nij", em[:, 1:], np.conj(em[:, 1:]))
    np.testing.assert_allclose(s, np.eye(3)[None] - np.einsum("ni,nj->nij", kh, kh), atol=1e-14)
