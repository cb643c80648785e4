"""Synthetic workloads of the hot path (parameters only, no arithmetic).

arXiv:2211.14056 benchmarks pp -> t tbar (g)(g) with real PDFs (Table 1,
Figs. 3-4); those inputs are not available, so these synthetic set-ups stand
in: a fixed partonic energy for g g -> t tbar, and a synthetic gluon
luminosity f(x) = x^-1.1 (1-x)^5 at sqrt(S) = 13 TeV for the 2 -> 3 and
2 -> 4 processes, with the cuts and widths below.  Dimension order: the two
luminosity uniforms (if any), then the RAMBO uniforms.
"""

PROCESS_IDS = {"gg_ttx": 1, "gg_ttxg": 2, "gg_ttxgg": 3, "uux_ttxgg": 4, "epem_mupmum": 5,
               "uxu_ttxgg": 6, "ug_ttxgu": 7, "gu_ttxgu": 8, "uxg_ttxgux": 9, "gux_ttxgux": 10}

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


# p p -> t t~ g g as the sum of its subprocesses (arXiv:2211.14056 Table 1),
# each channel a two-quark-line or gluon amplitude with its own Vegas grid and
# its parton pairs in the luminosity, from the synthetic tabulated set of
# ``pdfgrid`` (flavour index = PDG code + 4, gluon 4) at Q = sqrt(s_hat) / 2:
#   gg; q q~ and q~ q (q = d, u, s, c from beam 1 or 2); q g, g q, q~ g, g q~.
# Same energy, width and cuts as g g -> t t~ g g; the cuts apply to every final
# light parton (the gluon and the quark of the q g channels).
_PP = dict(mt=173.0, wt=1.5, gs=1.2177, sqrt_s=13000.0, lumi="pdf", mu_f=0.5, pt_cut=30.0, dr_cut=0.4,
           iterations=5)
PP_CHANNELS = {
    "pp_ttxgg_gg": dict(_PP, process="gg_ttxgg", pairs=[(4, 4)], events=2 ** 21, seed=11),
    "pp_ttxgg_qqx": dict(_PP, process="uux_ttxgg", pairs=[(5, 3), (6, 2), (7, 1), (8, 0)], events=2 ** 18, seed=12),
    "pp_ttxgg_qxq": dict(_PP, process="uxu_ttxgg", pairs=[(3, 5), (2, 6), (1, 7), (0, 8)], events=2 ** 18, seed=13),
    "pp_ttxgg_qg": dict(_PP, process="ug_ttxgu", pairs=[(5, 4), (6, 4), (7, 4), (8, 4)], events=2 ** 19, seed=14),
    "pp_ttxgg_gq": dict(_PP, process="gu_ttxgu", pairs=[(4, 5), (4, 6), (4, 7), (4, 8)], events=2 ** 19, seed=15),
    "pp_ttxgg_qxg": dict(_PP, process="uxg_ttxgux", pairs=[(3, 4), (2, 4), (1, 4), (0, 4)], events=2 ** 19, seed=16),
    "pp_ttxgg_gqx": dict(_PP, process="gux_ttxgux", pairs=[(4, 3), (4, 2), (4, 1), (4, 0)], events=2 ** 19, seed=17),
}
WORKLOADS.update(PP_CHANNELS)


# the batched mixed launch: four processes together, each with its own Vegas
# grid (the processes' own set-ups above), FP32 amplitudes
MIXED = {"workloads": ["gg_ttx_1tev", "gg_ttxg_13tev", "gg_ttxgg_13tev", "uux_ttxgg_13tev"],
         "events": [4_000_000, 1_000_000, 250_000, 10_000], "seed": 4}


def oracle_cfg(w):
    """The same workload as the keyword dict oracle.integrate.Setup takes
    (with tabulated densities: the synthetic set itself, the pairs, mu_f)."""
    keys = ("process", "mt", "wt", "gs", "sqrt_s", "lumi", "pt_cut", "dr_cut")
    cfg = {k: w[k] for k in keys}
    if w["lumi"] == "pdf":
        from .pdfgrid import synthetic_set
        cfg.update(pdf=synthetic_set(), pairs=list(w["pairs"]), mu_f=w["mu_f"])
    return cfg


def process_kwargs(w, precision, pdf=None):
    """Keyword arguments of binding.Process for a workload (pdf: the loaded
    set, a binding.PDFSet, for the tabulated-density workloads)."""
    kw = dict(mt=w["mt"], wt=w["wt"], gs=w["gs"], sqrt_s=w["sqrt_s"], lumi=w["lumi"],
              pt_cut=w["pt_cut"], dr_cut=w["dr_cut"], precision=precision)
    if w["lumi"] == "pdf":
        if pdf is None:
            raise ValueError("this workload needs a loaded parton-density set (pdf=)")
        kw.update(pdf=pdf, pairs=list(w["pairs"]), mu_f=w["mu_f"])
    return kw
