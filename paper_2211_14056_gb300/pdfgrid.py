"""A synthetic parton-density set: the tabulated input of the PDF interpolation.

arXiv:2211.14056 (Sec. 1) takes its parton densities from PDFFlow, which
interpolates tabulated LHAPDF sets; no such set is available here, so this
module writes one: x f(x, Q^2) for the flavours c~ s~ u~ d~ g d u s c on 97 x
41 nodes uniform in ln x (x from 1e-6 to 1) and ln Q^2 (Q^2 from 4 to 1e8
GeV^2), from smooth closed-form shapes with a mild ln Q^2 dependence (valence
quarks harden, sea and gluon steepen at small x as Q^2 grows; every density
vanishes at x = 1).  It is input data, like a file read from disk: it holds
none of the interpolation's arithmetic, and both the CUDA library and the
oracle receive the same table.

Flavour index of a parton with PDG code q: q + 4 for quarks (-4..4, without
0), 4 for the gluon (PDG 21).
"""
import numpy as np

X_MIN, X_MAX = 1e-6, 1.0
Q2_MIN, Q2_MAX = 4.0, 1e8
NX, NQ = 97, 41
FLAVOURS = ("cbar", "sbar", "ubar", "dbar", "g", "d", "u", "s", "c")
GLUON = 4


def index(pdg):
    """Flavour index of a PDG code (21 = gluon)."""
    if pdg == 21:
        return GLUON
    if pdg == 0 or abs(pdg) > 4:
        raise ValueError("flavours d, u, s, c, their antiquarks and the gluon")
    return pdg + 4


def nodes():
    """(x nodes [NX], Q^2 nodes [NQ])."""
    return (np.exp(np.linspace(np.log(X_MIN), np.log(X_MAX), NX)),
            np.exp(np.linspace(np.log(Q2_MIN), np.log(Q2_MAX), NQ)))


def synthetic_set():
    """dict(x_min, x_max, q2_min, q2_max, xf [9][NQ][NX] float64)."""
    x, q2 = nodes()
    X, Q2 = np.meshgrid(x, q2)                  # [NQ][NX]
    s = np.log(Q2 / Q2_MIN) / np.log(Q2_MAX / Q2_MIN)     # 0 .. 1
    om = 1.0 - X
    sea = 0.12 * X ** (-0.14 - 0.10 * s) * om ** (7.0 + 1.5 * s)
    ubar, dbar = sea, 1.15 * sea
    sbar = 0.55 * sea
    cbar = 0.25 * s * sea
    uv = 2.1 * X ** (0.55 + 0.05 * s) * om ** (3.0 + 0.6 * s)
    dv = 1.1 * X ** (0.60 + 0.05 * s) * om ** (4.0 + 0.6 * s)
    g = 1.9 * X ** (-0.08 - 0.18 * s) * om ** (5.0 + 1.2 * s)
    xf = np.stack([cbar, sbar, ubar, dbar, g, dv + dbar, uv + ubar, sbar, cbar])
    return {"x_min": X_MIN, "x_max": X_MAX, "q2_min": Q2_MIN, "q2_max": Q2_MAX, "xf": xf}
