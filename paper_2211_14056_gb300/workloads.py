"""Synthetic workloads of the hot path (parameters only, no arithmetic).

arXiv:2211.14056 benchmarks pp -> t tbar (g)(g) with real PDFs (Table 1,
Figs. 3-4); those inputs are not available, so these synthetic set-ups stand
in: a fixed partonic energy for g g -> t tbar, and a synthetic gluon
luminosity f(x) = x^-1.1 (1-x)^5 at sqrt(S) = 13 TeV for the 2 -> 3 and
2 -> 4 processes, with the cuts and widths below.  Dimension order: the two
luminosity uniforms (if any), then the RAMBO uniforms.
"""

PROCESS_IDS = {"gg_ttx": 1, "gg_ttxg": 2, "gg_ttxgg": 3, "uux_ttxgg": 4, "epem_mupmum": 5}

WORKLOADS = {
    # g g -> t tbar at fixed sqrt(s) = 1 TeV: closed-form target, FP64
    "gg_ttx_1tev": dict(process="gg_ttx", mt=173.0, wt=0.0, gs=1.2177, sqrt_s=1000.0, lumi=False,
                        pt_cut=0.0, dr_cut=0.0, events=65536, iterations=5, seed=1),
    # g g -> t tbar g with the synthetic luminosity and pT_g > 30 GeV
    "gg_ttxg_13tev": dict(process="gg_ttxg", mt=173.0, wt=0.0, gs=1.2177, sqrt_s=13000.0, lumi=True,
                          pt_cut=30.0, dr_cut=0.0, events=2 ** 20, iterations=10, seed=2),
    # g g -> t tbar g g, Gamma_t = 1.5 GeV, pT_g > 30 GeV and Delta R_gg > 0.4
    "gg_ttxgg_13tev": dict(process="gg_ttxgg", mt=173.0, wt=1.5, gs=1.2177, sqrt_s=13000.0, lumi=True,
                           pt_cut=30.0, dr_cut=0.4, events=2 ** 22, iterations=5, seed=3),
    # u u~ -> t t~ g g with the g g -> t t~ g g set-up (the luminosity serves u and u~)
    "uux_ttxgg_13tev": dict(process="uux_ttxgg", mt=173.0, wt=1.5, gs=1.2177, sqrt_s=13000.0, lumi=True,
                            pt_cut=30.0, dr_cut=0.4, events=10_000, iterations=5, seed=5),
    # e+ e- -> mu+ mu- (QED, photon exchange) at a fixed sqrt(s) = 100 GeV: closed-form
    # |M|^2 = e^4 (1 + cos^2 theta) and sigma = 4 pi alpha^2 / (3 s); mt and gs are unused
    "epem_mupmum_100gev": dict(process="epem_mupmum", mt=0.0, wt=0.0, gs=1.2177, sqrt_s=100.0, lumi=False,
                               pt_cut=0.0, dr_cut=0.0, events=2 ** 20, iterations=5, seed=6),
}


# the batched mixed launch: four processes together, each with its own Vegas
# grid (the processes' own set-ups above), FP32 amplitudes
MIXED = {"workloads": ["gg_ttx_1tev", "gg_ttxg_13tev", "gg_ttxgg_13tev", "uux_ttxgg_13tev"],
         "events": [4_000_000, 1_000_000, 250_000, 10_000], "seed": 4}


def oracle_cfg(w):
    """The same workload as the keyword dict oracle.integrate.Setup takes."""
    keys = ("process", "mt", "wt", "gs", "sqrt_s", "lumi", "pt_cut", "dr_cut")
    return {k: w[k] for k in keys}


def process_kwargs(w, precision):
    """Keyword arguments of binding.Process for a workload."""
    return dict(mt=w["mt"], wt=w["wt"], gs=w["gs"], sqrt_s=w["sqrt_s"], lumi=w["lumi"],
                pt_cut=w["pt_cut"], dr_cut=w["dr_cut"], precision=precision)
