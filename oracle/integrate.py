"""Event weights and Vegas iterations: the whole hot path, step by step.

Test infrastructure (see ``oracle/__init__``).

For one event with uniforms y[d] (arXiv:2211.14056, Sec. 1: tensorised Vegas
over events; the steps below follow the order in which the weight is built):

  1. x, J_vegas, bins = Vegas map of y                         (``vegas``)
  2. hadronic set-up: (x1, x2, s_hat, L) = luminosity map of x[0], x[1]
     (a synthetic gluon density, or tabulated densities summed over the
     channel's parton pairs, ``pdf``);
     fixed partonic set-up: s_hat = s, L = 1                   (``phase_space``)
  3. massless momenta and Phi_n from the remaining x           (RAMBO on diet)
  4. massive momenta and weight factor W                       (rescaling)
  5. cut indicator on the final gluons
  6. |M|^2 of the partonic momenta (CM frame, beam 1 along +z) (``processes``)
  7. w = |M|^2 Phi_n W J_vegas L / (2 s_hat) * 0.3893793721e9 pb GeV^2 * cut

Dimension order: (x_a, x_b) of the luminosity map when it is on, then the
n-2 RAMBO mass uniforms, then n-1 (cos theta, phi) pairs.
"""
import math
import numpy as np

from . import philox, vegas, phase_space as ps
from .processes import Process, final_jets
from .pdf import PDFGrid
from .berends_giele import QQbarGluons


def n_final(name):
    from .processes import PROCESSES
    return len(PROCESSES[name][0]) - 2


def ndim(cfg):
    n = n_final(cfg["process"])
    return 3 * n - 4 + (2 if cfg.get("lumi", False) else 0)


class Setup:
    """One configured integrand: process, energies, luminosity, cuts."""

    def __init__(self, cfg, amplitude="feynman"):
        self.cfg = dict(cfg)
        self.name = cfg["process"]
        self.proc = Process(self.name, mt=cfg.get("mt", 173.0), wt=cfg.get("wt", 0.0),
                            gs=cfg.get("gs", 1.2177))
        self.n = n_final(self.name)
        self.ndim = ndim(cfg)
        self.lumi = cfg.get("lumi", False)
        self.masses = [self.proc.mass.get(x, 0.0) for x in self.proc.particles[2:]]
        self.gluons = final_jets(self.name)       # the cuts' partons: final gluons and light quarks
        self.pdf = None
        if self.lumi == "pdf":
            d = cfg["pdf"]
            self.pdf = PDFGrid(d["x_min"], d["x_max"], d["q2_min"], d["q2_max"], d["xf"])
        self.bg = QQbarGluons(self.proc) if amplitude == "bg" else None

    def kinematics(self, y, edges):
        """Steps 1-5: (momenta [N, n+2, 4], weight without |M|^2 [N], bins, cut)."""
        c = self.cfg
        x, jac, bins = vegas.vegas_map(y, edges)
        if self.lumi == "pdf":
            S = c["sqrt_s"] ** 2
            tau0 = (sum(self.masses)) ** 2 / S
            x1, x2, shat, L = ps.pdf_luminosity_map(x[0], x[1], tau0, S, self.pdf, c["pairs"], c.get("mu_f", 0.5))
            xr = x[2:]
        elif self.lumi:
            S = c["sqrt_s"] ** 2
            tau0 = (sum(self.masses)) ** 2 / S
            x1, x2, shat, L = ps.luminosity_map(x[0], x[1], tau0, S,
                                                c.get("lumi_N", 1.0), c.get("lumi_a", -1.1),
                                                c.get("lumi_b", 5.0))
            xr = x[2:]
        else:
            shat = np.full(y.shape[1], c["sqrt_s"] ** 2)
            L = np.ones(y.shape[1])
            xr = x
        rs = np.sqrt(shat)
        pm, wps = ps.rambo_diet(rs, xr, self.n)
        k, wm = ps.massive(pm, self.masses, rs)
        N = y.shape[1]
        p = np.zeros((N, self.n + 2, 4))
        p[:, 0, 0] = p[:, 0, 3] = rs / 2
        p[:, 1, 0] = rs / 2
        p[:, 1, 3] = -rs / 2
        p[:, 2:] = k
        cut = ps.pass_cuts(p, self.gluons, c.get("pt_cut", 0.0), c.get("dr_cut", 0.0))
        wk = wps * wm * jac * L / (2.0 * shat) * ps.GEV2_TO_PB * cut
        return p, wk, bins, cut

    def me2(self, p):
        if self.bg is not None:
            return self.bg.me2(p)
        return self.proc.me2_batched(p)

    def weights(self, y, edges):
        """Step 7: w [N] and bins [d, N]; |M|^2 is evaluated only where the
        cut indicator is 1 (elsewhere w = 0 whatever |M|^2 is)."""
        p, wk, bins, cut = self.kinematics(y, edges)
        w = np.zeros(y.shape[1])
        if np.any(cut):
            w[cut] = self.me2(p[cut]) * wk[cut]
        return w, bins


def iteration(setup, seed, it, nev, edges, events=None):
    """One Vegas iteration over global events 0..nev-1 (or the listed ones).

    Returns dict(I, var, sum_w, sum_w2, hist, w, bins).
    """
    ev = np.arange(nev, dtype=np.uint64) if events is None else np.asarray(events, dtype=np.uint64)
    y = philox.uniforms(seed, it, ev, setup.ndim)
    w, bins = setup.weights(y, edges)
    sw, sw2, hist = vegas.accumulate(w, bins, edges.shape[1] - 1)
    I, var = vegas.estimate(sw, sw2, ev.size)
    return dict(I=I, var=var, sum_w=sw, sum_w2=sw2, hist=hist, w=w, bins=bins)


def integrate(setup, seed, iterations, nev, edges=None, refine_last=False):
    """Iterations 0..iterations-1 with refinement after each one (but the
    last unless ``refine_last``); returns (results, final edges, combined)."""
    if edges is None:
        edges = vegas.uniform_grid(setup.ndim)
    results = []
    for it in range(iterations):
        r = iteration(setup, seed, it, nev, edges)
        results.append(r)
        if it < iterations - 1 or refine_last:
            edges = vegas.refine(edges, r["hist"])
    comb = vegas.combine([r["I"] for r in results], [r["var"] for r in results])
    return results, edges, comb
