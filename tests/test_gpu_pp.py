"""GPU: tabulated parton densities and the subprocess sum of p p -> t t~ g g.

* mf_pdf_eval (the interpolation kernel) against the oracle's log-bicubic
  interpolation of the same table: FP64 to 1e-12 relative, FP32 to 5e-5 of
  the value at worst and 1e-6 at the median (with an absolute floor where a
  density vanishes: near x -> 1 the value is a small difference of node values
  and slopes, ~200 ulps of FP32),
  at ragged sizes, at the table's nodes and edges and outside its range;
* each crossed subprocess (q~ q, q g, g q, q~ g, g q~ -> t t~ g + jet) per
  event against the oracle's Feynman diagrams for that flavour list
  (assert_fp64_parity, its tail arbitrated by the oracle's spread);
* Vegas iterations of each channel with the tabulated-density luminosity
  (sum over the channel's parton pairs) against the oracle: weights, I_k,
  sigma_k, the refined grid;
* the seven channels in one mixed launch equal their separate iterations.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import integrate as oi, philox as oph, vegas as ov  # noqa: E402
from oracle.pdf import PDFGrid  # noqa: E402
from tests.test_gpu_parity import _aos_to_soa, assert_fp64_parity  # noqa: E402

pytestmark = pytest.mark.gpu

CHANNELS = ["pp_ttxgg_gg", "pp_ttxgg_qqx", "pp_ttxgg_qxq", "pp_ttxgg_qg", "pp_ttxgg_gq", "pp_ttxgg_qxg",
            "pp_ttxgg_gqx"]


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14056_gb300 as mf
    return mf


@pytest.fixture(scope="module")
def pdf(mf):
    from paper_2211_14056_gb300.pdfgrid import synthetic_set
    return mf.PDFSet.from_dict(synthetic_set())


def _oracle_pdf():
    from paper_2211_14056_gb300.pdfgrid import synthetic_set
    d = synthetic_set()
    return PDFGrid(d["x_min"], d["x_max"], d["q2_min"], d["q2_max"], d["xf"]), d


def _proc(mf, pdf, name, precision, **over):
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = dict(WORKLOADS[name], **over)
    return mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, precision, pdf=pdf)), w


def _setup(w, amplitude="feynman"):
    from paper_2211_14056_gb300.workloads import oracle_cfg
    return oi.Setup(oracle_cfg(w), amplitude=amplitude)


def _points(n, seed):
    from paper_2211_14056_gb300 import pdfgrid
    rng = np.random.default_rng(seed)
    lx = rng.uniform(np.log(pdfgrid.X_MIN) - 1.0, 0.0, n)           # some below the table
    lq = rng.uniform(np.log(pdfgrid.Q2_MIN) - 1.0, np.log(pdfgrid.Q2_MAX) + 1.0, n)
    x, q2 = np.exp(lx), np.exp(lq)
    xn, qn = pdfgrid.nodes()
    m = min(40, n)
    x[:m] = xn[rng.integers(0, len(xn), m)]                          # nodes, including x = 1
    q2[:m] = qn[rng.integers(0, len(qn), m)]
    return x, q2


def _lumi_spread(st, y, edges):
    """Relative FP64 rounding of the tabulated-density luminosity of the
    events with uniforms y[:, e]: the oracle's FP64 value against the same
    scheme in extended precision, plus the change one ulp of x1, x2 or Q^2
    makes (near x -> 1 a density is a small difference of its node values and
    slopes, and its relative rounding grows to ~1e-12)."""
    from oracle import phase_space as ps
    x, _, _ = ov.vegas_map(y, edges)
    c = st.cfg
    S = c["sqrt_s"] ** 2
    tau0 = (sum(st.masses)) ** 2 / S
    x1 = tau0 ** x[0]
    x2 = (tau0 / x1) ** x[1]
    q2 = c["mu_f"] ** 2 * x1 * x2 * S
    d = c["pdf"]
    ext = PDFGrid(d["x_min"], d["x_max"], d["q2_min"], d["q2_max"], d["xf"], dtype=np.longdouble)

    def lum(g, a1, a2, q):
        return sum(g.xfx(fa, a1, q) * g.xfx(fb, a2, q) for fa, fb in c["pairs"])

    X = [np.asarray(v, dtype=np.longdouble) for v in (x1, x2, q2)]
    le = lum(ext, *X)
    spread = np.abs(lum(st.pdf, x1, x2, q2) - le)
    for k in range(3):
        Xk = list(X)
        Xk[k] = Xk[k] * (1 + np.longdouble(2.0 ** -52))
        spread = spread + np.abs(lum(ext, *Xk) - le)
    return np.asarray(spread / np.abs(le), dtype=np.float64)


@pytest.mark.parametrize("n", [10007, 1, 0])
def test_pdf_eval_matches_oracle(mf, pdf, n):
    og, d = _oracle_pdf()
    x, q2 = _points(max(n, 1), seed=n)
    x, q2 = x[:n], q2[:n]
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    qt = torch.tensor(q2, dtype=torch.float64, device="cuda")
    for f in range(9):
        ref = og.xfx(f, x, q2) if n else np.zeros(0)
        for prec, bar in ((mf.MF_FP64, 1e-12), (mf.MF_FP32, 5e-5)):
            out = torch.full((max(n, 1),), float("nan"), dtype=torch.float64, device="cuda")
            pdf.eval(f, n, xt, qt, out, precision=prec)
            torch.cuda.synchronize()
            if n == 0:
                continue
            got = out[:n].cpu().numpy()
            # FP32: a density that vanishes linearly (charm at the lowest Q^2,
            # every flavour at x -> 1) is compared against 1e-3 of its table's
            # scale there
            floor = 1e-6 if prec == mf.MF_FP64 else 1e-3
            scale = np.maximum(np.abs(ref), floor * np.max(np.abs(d["xf"][f])))
            err = np.abs(got - ref) / scale
            assert err.max() < bar, (f, prec, err.max())
            assert np.median(err) < (1e-14 if prec == mf.MF_FP64 else 1e-6)


def test_pdf_eval_over_several_passes_matches_oracle(mf, pdf):
    """A launch whose threads take several passes over the points (the
    persistent grid holds about half a million points per pass) with a ragged
    last pass: every point against the oracle, in FP64 and FP32, for the
    gluon and a quark flavour."""
    from paper_2211_14056_gb300 import pdfgrid
    og, d = _oracle_pdf()
    n = 1_500_007
    x, q2 = _points(n, seed=11)
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    qt = torch.tensor(q2, dtype=torch.float64, device="cuda")
    for f in (pdfgrid.GLUON, 1):
        ref = og.xfx(f, x, q2)
        for prec, bar in ((mf.MF_FP64, 1e-12), (mf.MF_FP32, 5e-5)):
            out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            pdf.eval(f, n, xt, qt, out, precision=prec)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            floor = 1e-6 if prec == mf.MF_FP64 else 1e-3
            scale = np.maximum(np.abs(ref), floor * np.max(np.abs(d["xf"][f])))
            err = np.abs(got - ref) / scale
            assert err.max() < bar, (f, prec, err.max())


def test_pdf_eval_arguments(mf, pdf):
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(mf.MFError):
        pdf.eval(9, 4, x, x, x)
    with pytest.raises(mf.MFError):
        pdf.eval(0, 4, x, x, x, precision=mf.MF_FP32_TC)
    with pytest.raises(mf.MFError):
        mf.PDFSet(1e-3, 1.0, 1.0, 10.0, np.ones((1, 3, 10)))        # too few Q^2 nodes


def _events(st, seed, nev):
    y = oph.uniforms(seed, 0, np.arange(6 * nev, dtype=np.uint64), st.ndim)
    po, _, _, cut = st.kinematics(y, ov.uniform_grid(st.ndim))
    return po[cut][:nev]


@pytest.mark.parametrize("name", CHANNELS[1:])
def test_channel_matrix_element_matches_oracle(mf, pdf, name):
    p, w = _proc(mf, pdf, name, mf.MF_FP64)
    st = _setup(w)
    po = _events(st, 3, 60)
    assert len(po) == 60
    ref = st.proc.me2_batched(po)
    out = torch.empty(len(po), dtype=torch.float64, device="cuda")
    p.matrix_element(len(po), _aos_to_soa(po), out)
    torch.cuda.synchronize()
    assert_fp64_parity(out.cpu().numpy(), ref, momenta=po, setup=st)
    p32, _ = _proc(mf, pdf, name, mf.MF_FP32)
    p32.matrix_element(len(po), _aos_to_soa(po), out)
    torch.cuda.synchronize()
    rel = np.abs(out.cpu().numpy() / ref - 1)
    print(f"{name} FP32 |M|^2: median {np.median(rel):.1e} max {rel.max():.1e}")
    assert np.median(rel) < 1e-5 and rel.max() < 5e-3


@pytest.mark.parametrize("name,n", [("pp_ttxgg_gg", 400), ("pp_ttxgg_qqx", 500), ("pp_ttxgg_qg", 500),
                                    ("pp_ttxgg_gqx", 500)])
def test_channel_iterations_match_oracle(mf, pdf, name, n):
    """Two refined iterations per channel on the tabulated-density
    luminosity, each compared on the GPU's own current edges; a weight outside
    1e-12 is held to the oracle's spread of |M|^2 plus the FP64 rounding of
    the luminosity at that event."""
    p, w = _proc(mf, pdf, name, mf.MF_FP64)
    g = p.grid()
    st = _setup(w, amplitude="bg" if w["process"] == "gg_ttxgg" else "feynman")
    wt = torch.empty(n, dtype=torch.float64, device="cuda")
    for it in range(2):
        edges = g.get()
        r = p.vegas_iterate(g, seed=19, it=it, n=n, refine=True, weights=wt)
        ro = oi.iteration(st, 19, it, n, edges)
        wg = wt.cpu().numpy()
        np.testing.assert_array_equal(wg > 0, ro["w"] > 0)
        nz = ro["w"] > 0
        assert nz.sum() > 0.3 * n
        y = oph.uniforms(19, it, np.arange(n, dtype=np.uint64), st.ndim)
        pk = st.kinematics(y, edges)[0]
        yz = y[:, nz]
        allowed = assert_fp64_parity(wg[nz], ro["w"][nz], tail=1e-9, momenta=pk[nz], setup=st,
                                     extra=lambda idx: _lumi_spread(st, yz[:, idx], edges))
        # the estimate and its error may move by what the events were allowed
        wo = np.abs(ro["w"][nz])
        bound_I = 1e-12 + np.sum(allowed * wo) / np.sum(wo)
        bound_s = 1e-11 + 2 * np.sum(allowed * wo * wo) / np.sum(wo * wo)
        print(f"{name} it {it}: I_k {abs(r['I_k'] / ro['I'] - 1):.1e} (bound {bound_I:.1e})")
        assert r["I_k"] == pytest.approx(ro["I"], rel=bound_I)
        assert r["sigma_k"] == pytest.approx(math.sqrt(ro["var"]), rel=bound_s)
        # the refined edges: the histogram of w^2 may move, bin by bin, by what
        # its events were allowed (twice the weights' relative allowance), and
        # an edge by at most that relative change (edges lie in [0, 1])
        w2 = ro["w"] ** 2
        a = np.zeros(n)
        a[nz] = allowed
        dev = 0.0
        for j in range(st.ndim):
            num = np.bincount(ro["bins"][j], weights=2 * a * w2, minlength=edges.shape[1] - 1)
            den = np.bincount(ro["bins"][j], weights=w2, minlength=edges.shape[1] - 1)
            dev = max(dev, np.max(num[den > 0] / den[den > 0]))
        np.testing.assert_allclose(g.get(), ov.refine(edges, ro["hist"]), rtol=0, atol=1e-12 + dev)


@pytest.mark.parametrize("precision,tile,bar", [(0, 0, 1e-12), (1, 32, 1e-6), (1, 0, 1e-12)])
def test_seven_channels_in_one_mixed_launch(mf, pdf, precision, tile, bar):
    """FP64 with the per-process form (seven FP64 processes' sums do not fit
    beside the shared queue's stores: that form is refused); FP32 with the
    shared queue (the queue's |M|^2 code path, ~1e-7 from the process's own
    kernel in FP32) and the per-process form (the same kernels: to rounding
    of the sums)."""
    procs = [_proc(mf, pdf, name, precision)[0] for name in CHANNELS]
    n = [3000, 800, 800, 1500, 1500, 1500, 1500]
    mg = [p.grid() for p in procs]
    sg = [p.grid() for p in procs]
    mx = mf.Mixed(procs, mg, n)
    if precision == 0:
        with pytest.raises(mf.MFError):
            mx.set_launch(0, 32)
    mx.set_launch(0, tile)
    for it in range(2):
        res = mx.run(seed=23, it=it, refine=True)
        for k, p in enumerate(procs):
            ref = p.vegas_iterate(sg[k], 23, it, n[k], refine=True)
            assert res[k]["n_pass"] == ref["n_pass"] > 0
            assert res[k]["I_k"] == pytest.approx(ref["I_k"], rel=bar)
            np.testing.assert_allclose(mg[k].get(), sg[k].get(), rtol=0, atol=max(bar, 1e-12))


def test_unsupported_paths(mf, pdf):
    p, _ = _proc(mf, pdf, "pp_ttxgg_gg", mf.MF_FP64)
    with pytest.raises(mf.MFError):
        p.grad(p.grid(), 1, 0, 10)
    with pytest.raises(mf.MFError):
        _proc(mf, pdf, "pp_ttxgg_qg", mf.MF_FP32_TC)
