"""External wavefunctions: helicity spinors and gluon/photon polarisation vectors.

Test infrastructure (see ``oracle/__init__``).

The paper (arXiv:2211.14056, Sec. 2, Fig. 2) evaluates MadGraph's
``wavefunctions.py``: HELAS external states (H. Murayama, I. Watanabe,
K. Hagiwara, KEK-91-11).  Conventions written out here:

* chiral (Weyl) representation: gamma^0 = [[0, 1], [1, 0]],
  gamma^k = [[0, sigma^k], [-sigma^k, 0]]; spinors are (psi_L, psi_R);
* two-component helicity eigenstates of the direction p/|p|,
      chi_+ = (|p| + p_z, p_x + i p_y) / sqrt(2|p|(|p| + p_z)),
      chi_- = (-p_x + i p_y, |p| + p_z) / sqrt(2|p|(|p| + p_z)),
  with the limits chi_+ = (0, 1), chi_- = (-1, 0) for p along -z and the
  +z states for |p| = 0;
* u(p, l) = (w_{-l} chi_l, w_l chi_l),  v(p, l) = (-l w_l chi_{-l}, l w_{-l} chi_{-l}),
  w_(+-) = sqrt(E +- |p|) (massless: w_+ = sqrt(2E), w_- = 0), helicity
  l = +-1 (twice the spin projection);
* massless vector: eps(k, l) = (-l e1 - i e2)/sqrt(2), with e1, e2 the unit
  vectors along theta and phi of k (for k_T = 0 the phi = 0 limit).

Every external state of a helicity sum only has to satisfy the Dirac equation,
completeness (sum u ubar = p-slash + m, sum v vbar = p-slash - m) and
transversality; those are what the tests check.
"""
import numpy as np

I2 = np.eye(2, dtype=complex)
SIGMA = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=complex)
GAMMA = np.zeros((4, 4, 4), dtype=complex)
GAMMA[0, :2, 2:] = I2
GAMMA[0, 2:, :2] = I2
for _k in range(3):
    GAMMA[_k + 1, :2, 2:] = SIGMA[_k]
    GAMMA[_k + 1, 2:, :2] = -SIGMA[_k]
METRIC = np.diag([1.0, -1.0, -1.0, -1.0])


def mdot(a, b):
    """Minkowski product a.b over the last axis (no complex conjugation)."""
    return a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1] - a[..., 2] * b[..., 2] - a[..., 3] * b[..., 3]


def slash(v):
    """gamma^mu v_mu as [..., 4, 4] for contravariant components v[..., 4]."""
    v_low = v * METRIC.diagonal()
    return np.einsum("...m,mab->...ab", v_low, GAMMA)


def _chi(p3, lam):
    """Two-component helicity eigenstates [N, 2] of directions p3 [N, 3]."""
    px, py, pz = p3[:, 0], p3[:, 1], p3[:, 2]
    pa = np.sqrt(px * px + py * py + pz * pz)
    s = pa + pz
    out = np.zeros((p3.shape[0], 2), dtype=complex)
    regular = s > 0
    norm = np.sqrt(2.0 * pa * s, where=regular, out=np.ones_like(s))
    if lam > 0:
        out[:, 0] = np.where(regular, s / norm, 0.0)
        out[:, 1] = np.where(regular, (px + 1j * py) / norm, 1.0)
    else:
        out[:, 0] = np.where(regular, (-px + 1j * py) / norm, -1.0)
        out[:, 1] = np.where(regular, s / norm, 0.0)
    rest = pa == 0
    if np.any(rest):
        out[rest] = [1.0, 0.0] if lam > 0 else [0.0, 1.0]
    return out


def _omegas(p, mass):
    """(sqrt(E + |p|), sqrt(E - |p|)); for mass 0 the second is 0 exactly."""
    pa = np.sqrt(np.sum(p[:, 1:] ** 2, axis=1))
    E = p[:, 0]
    if mass == 0:
        return np.sqrt(2.0 * E), np.zeros_like(E)
    return np.sqrt(np.maximum(E + pa, 0.0)), np.sqrt(np.maximum(E - pa, 0.0))


def u_spinor(p, mass, lam):
    """Dirac u(p, lam) [N, 4] (column)."""
    wp, wm = _omegas(p, mass)
    chi = _chi(p[:, 1:], lam)
    w_l, w_ml = (wp, wm) if lam > 0 else (wm, wp)
    return np.concatenate([w_ml[:, None] * chi, w_l[:, None] * chi], axis=1)


def v_spinor(p, mass, lam):
    """Dirac v(p, lam) [N, 4] (column)."""
    wp, wm = _omegas(p, mass)
    chi = _chi(p[:, 1:], -lam)
    w_l, w_ml = (wp, wm) if lam > 0 else (wm, wp)
    return np.concatenate([-lam * w_l[:, None] * chi, lam * w_ml[:, None] * chi], axis=1)


def bar(psi):
    """Dirac adjoint psi^dagger gamma^0 as a row spinor [..., 4]."""
    return np.einsum("...a,ab->...b", np.conj(psi), GAMMA[0])


def polarisation(k, lam):
    """Massless polarisation vector eps(k, lam) [N, 4] (contravariant)."""
    kx, ky, kz = k[:, 1], k[:, 2], k[:, 3]
    kt = np.sqrt(kx * kx + ky * ky)
    ka = np.sqrt(kt * kt + kz * kz)
    e1 = np.zeros((k.shape[0], 4))
    e2 = np.zeros((k.shape[0], 4))
    reg = kt > 0
    ktr = np.where(reg, kt, 1.0)
    e1[:, 1] = np.where(reg, kx * kz / (ka * ktr), np.sign(kz))
    e1[:, 2] = np.where(reg, ky * kz / (ka * ktr), 0.0)
    e1[:, 3] = np.where(reg, -kt / ka, 0.0)
    e2[:, 1] = np.where(reg, -ky / ktr, 0.0)
    e2[:, 2] = np.where(reg, kx / ktr, 1.0)
    return (-lam * e1 - 1j * e2) / np.sqrt(2.0)
