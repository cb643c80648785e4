"""GPU: u u~ -> t t~ g g (two quark lines; generated Feynman-diagram code with
its colour decomposition) against the oracle's explicit-colour Feynman sum,
per event and through Vegas iterations, and inside the mixed launch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle.integrate as oi
import oracle.philox as oph
import oracle.vegas as ov
from tests.test_gpu_parity import _aos_to_soa, assert_fp64_parity

pytestmark = pytest.mark.gpu

NAME = "uux_ttxgg_13tev"


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14056_gb300 as mf
    return mf


def _proc(mf, precision, name=NAME, **over):
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = dict(WORKLOADS[name], **over)
    return mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, precision)), w


def _setup(w):
    from paper_2211_14056_gb300.workloads import oracle_cfg
    return oi.Setup(oracle_cfg(w))


def _events(st, seed, nev):
    y = oph.uniforms(seed, 0, np.arange(4 * nev, dtype=np.uint64), st.ndim)
    po, _, _, cut = st.kinematics(y, ov.uniform_grid(st.ndim))
    return po[cut][:nev]


@pytest.mark.parametrize("wt", [0.0, 1.5])
def test_matrix_element_fp64_matches_oracle(mf, wt):
    p, w = _proc(mf, mf.MF_FP64, wt=wt)
    st = _setup(w)
    po = _events(st, 3, 120)
    ref = st.proc.me2_batched(po)
    out = torch.empty(len(po), dtype=torch.float64, device="cuda")
    p.matrix_element(len(po), _aos_to_soa(po), out)
    torch.cuda.synchronize()
    assert_fp64_parity(out.cpu().numpy(), ref, momenta=po, setup=st)


def test_matrix_element_fp32_error(mf):
    p, w = _proc(mf, mf.MF_FP32)
    st = _setup(w)
    po = _events(st, 4, 120)
    ref = st.proc.me2_batched(po)
    out = torch.empty(len(po), dtype=torch.float64, device="cuda")
    p.matrix_element(len(po), _aos_to_soa(po), out)
    torch.cuda.synchronize()
    rel = np.abs(out.cpu().numpy() / ref - 1)
    print(f"u u~ -> t t~ g g FP32 |M|^2 rel. error: max {rel.max():.2e} median {np.median(rel):.2e}")
    assert np.median(rel) < 1e-5 and np.quantile(rel, 0.99) < 1e-3 and rel.max() < 5e-3


def test_vegas_iterations_match_oracle(mf):
    """Two refined iterations.  The refined edges agree with the oracle's to
    1e-12 absolute (the GPU sums the damped weights in a scan order); a bin
    width is ~1/50, so that rounding moves a Jacobian by up to ~1e-11
    relative, and each iteration is compared on the GPU's own edges."""
    p, w = _proc(mf, mf.MF_FP64)
    g = p.grid()
    st = _setup(w)
    edges = ov.uniform_grid(st.ndim)
    n = 1000
    wt = torch.empty(n, dtype=torch.float64, device="cuda")
    for it in range(2):
        r = p.vegas_iterate(g, seed=9, it=it, n=n, refine=True, weights=wt)
        ro = oi.iteration(st, 9, it, n, edges)
        wg = wt.cpu().numpy()
        np.testing.assert_array_equal(wg > 0, ro["w"] > 0)
        nz = ro["w"] > 0
        pk = st.kinematics(oph.uniforms(9, it, np.arange(n, dtype=np.uint64), st.ndim), edges)[0]
        assert_fp64_parity(wg[nz], ro["w"][nz], momenta=pk[nz], setup=st)
        assert r["I_k"] == pytest.approx(ro["I"], rel=1e-10)
        assert r["sigma_k"] == pytest.approx(np.sqrt(ro["var"]), rel=1e-9)
        np.testing.assert_allclose(g.get(), ov.refine(edges, ro["hist"]), rtol=0, atol=1e-12)
        edges = g.get()


def test_unsupported_paths_and_sizes(mf):
    p, w = _proc(mf, mf.MF_FP64)
    g = p.grid()
    with pytest.raises(mf.MFError):
        p.grad(g, 1, 0, 10)
    with pytest.raises(mf.MFError):
        _proc(mf, mf.MF_FP32_TC)
    edges = torch.tensor(g.get(), dtype=torch.float64, device="cuda").contiguous()
    totals = torch.empty(2 + p.ndim * 50 + 2, dtype=torch.float64, device="cuda")
    with pytest.raises(mf.MFError):
        p.vegas_accumulate_static(edges.view(-1), 50, 1, 0, 0, 10, totals)
    # one event and a ragged count
    st = _setup(w)
    po = _events(st, 6, 37)
    ref = st.proc.me2_batched(po)
    out = torch.empty(37, dtype=torch.float64, device="cuda")
    p.matrix_element(37, _aos_to_soa(po), out)
    one = torch.empty(1, dtype=torch.float64, device="cuda")
    p.matrix_element(1, _aos_to_soa(po[:1]), one)
    torch.cuda.synchronize()
    assert_fp64_parity(out.cpu().numpy(), ref, momenta=po, setup=st)
    assert one.item() == out[0].item()


@pytest.mark.parametrize("tile", [32, 0])
def test_mixed_with_four_processes(mf, tile):
    """The C4 mix (three gluon-initiated processes and u u~ -> t t~ g g): the
    mixed launch gives each process its own iteration's result (FP64)."""
    from paper_2211_14056_gb300.workloads import MIXED
    procs = []
    for name in MIXED["workloads"]:
        procs.append(_proc(mf, mf.MF_FP64, name=name)[0])
    n = [4000, 2000, 600, 600]
    mg = [p.grid() for p in procs]
    sg = [p.grid() for p in procs]
    mx = mf.Mixed(procs, mg, n)
    mx.set_launch(0, tile)
    for it in range(2):
        res = mx.run(seed=21, it=it, refine=True)
        for k, p in enumerate(procs):
            ref = p.vegas_iterate(sg[k], 21, it, n[k], refine=True)
            assert res[k]["n_pass"] == ref["n_pass"]
            assert res[k]["I_k"] == pytest.approx(ref["I_k"], rel=1e-12)
            np.testing.assert_allclose(mg[k].get(), sg[k].get(), rtol=0, atol=1e-12)
