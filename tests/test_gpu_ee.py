"""GPU: e+ e- -> mu+ mu- (QED, one s-channel photon diagram) against the
oracle's Feynman-diagram sum and the textbook closed forms
|M|^2 = e^4 (1 + cos^2 theta) and sigma = 4 pi alpha^2 / (3 s), per event,
through the sampler, through refined Vegas iterations and inside the mixed
launch."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle.integrate as oi
import oracle.philox as oph
import oracle.vegas as ov
from oracle.phase_space import GEV2_TO_PB
from tests.test_gpu_parity import _aos_to_soa, _soa_to_aos, assert_fp64_parity, random_grid

pytestmark = pytest.mark.gpu

NAME = "epem_mupmum_100gev"


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
    y = oph.uniforms(seed, 0, np.arange(nev, dtype=np.uint64), st.ndim)
    return st.kinematics(y, ov.uniform_grid(st.ndim))[0]


def _axis_events(rs):
    """mu- along +z, -z and +x (cos theta = 1, -1, 0): the limiting form of
    the helicity spinors on the z axis."""
    E = rs / 2
    out = []
    for d in ([0, 0, 1], [0, 0, -1], [1, 0, 0]):
        k = E * np.array(d, dtype=float)
        out.append([[E, 0, 0, E], [E, 0, 0, -E], [E, *k], [E, *(-k)]])
    return np.array(out)


def test_matrix_element_matches_closed_form_and_oracle(mf):
    p, w = _proc(mf, mf.MF_FP64)
    st = _setup(w)
    po = np.concatenate([_events(st, 3, 500), _axis_events(w["sqrt_s"])])
    out = torch.empty(len(po), dtype=torch.float64, device="cuda")
    p.matrix_element(len(po), _aos_to_soa(po), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    cos = po[:, 2, 3] / po[:, 2, 0]
    e = st.proc.ee
    np.testing.assert_allclose(got, e ** 4 * (1 + cos ** 2), rtol=1e-13)
    assert_fp64_parity(got, st.proc.me2_batched(po), core=1e-13, tail=1e-12, frac=1.0)


def test_matrix_element_fp32_error(mf):
    p, w = _proc(mf, mf.MF_FP32)
    st = _setup(w)
    po = _events(st, 4, 500)
    out = torch.empty(len(po), dtype=torch.float64, device="cuda")
    p.matrix_element(len(po), _aos_to_soa(po), out)
    torch.cuda.synchronize()
    rel = np.abs(out.cpu().numpy() / st.proc.me2_batched(po) - 1)
    assert rel.max() < 1e-5


def test_sample_matches_oracle(mf):
    """RAMBO with two massless final particles (the rescaling is the identity,
    xi = 1): momenta, phase-space weights and bins of the sampler."""
    p, w = _proc(mf, mf.MF_FP64)
    g = p.grid()
    edges = random_grid(p.ndim, seed=12)
    g.set(edges)
    n = 2049
    mom = torch.empty(p.n_ext * 4 * n, dtype=torch.float64, device="cuda")
    wps = torch.empty(n, dtype=torch.float64, device="cuda")
    bins = torch.empty(p.ndim * n, dtype=torch.uint8, device="cuda")
    p.sample(g, seed=78, it=2, n=n, momenta=mom, weight_ps=wps, bins=bins)
    torch.cuda.synchronize()
    st = _setup(w)
    y = oph.uniforms(78, 2, np.arange(n, dtype=np.uint64), st.ndim)
    po, wk, bo, cut = st.kinematics(y, edges)
    assert cut.all()
    np.testing.assert_array_equal(bins.view(p.ndim, n).cpu().numpy(), bo)
    pg = _soa_to_aos(mom, p.n_ext, n)
    assert np.max(np.abs(pg - po)) / w["sqrt_s"] < 1e-13
    np.testing.assert_allclose(wps.cpu().numpy(), wk, rtol=1e-13)


def test_vegas_iterations_match_oracle(mf):
    p, w = _proc(mf, mf.MF_FP64)
    g = p.grid()
    st = _setup(w)
    edges = ov.uniform_grid(st.ndim)
    n = 3000
    wt = torch.empty(n, dtype=torch.float64, device="cuda")
    for it in range(2):
        r = p.vegas_iterate(g, seed=9, it=it, n=n, refine=True, weights=wt)
        ro = oi.iteration(st, 9, it, n, edges)
        assert_fp64_parity(wt.cpu().numpy(), ro["w"], core=1e-13, tail=1e-11, frac=0.99)
        assert r["n_pass"] == n
        assert r["I_k"] == pytest.approx(ro["I"], rel=1e-12)
        assert r["sigma_k"] == pytest.approx(np.sqrt(ro["var"]), rel=1e-9)
        np.testing.assert_allclose(g.get(), ov.refine(edges, ro["hist"]), rtol=0, atol=1e-12)
        edges = g.get()


@pytest.mark.parametrize("precision", ["MF_FP64", "MF_FP32"])
def test_cross_section_closed_form(mf, precision):
    """Five refined iterations of 2^20 events: the combined estimate agrees
    with 4 pi alpha^2 / (3 s) within 4 standard errors, and that error is
    below 1e-4 relative."""
    p, w = _proc(mf, getattr(mf, precision))
    g = p.grid()
    for it in range(w["iterations"]):
        r = p.vegas_iterate(g, seed=w["seed"], it=it, n=w["events"], refine=True)
    alpha = 1.0 / 137.035999
    ref = 4 * math.pi * alpha ** 2 / (3 * w["sqrt_s"] ** 2) * GEV2_TO_PB
    print(f"e+e- -> mu+mu- ({precision}): {r['I']:.8f} +- {r['sigma']:.2e} pb, closed form {ref:.8f} pb")
    assert abs(r["I"] - ref) < 4 * r["sigma"]
    assert r["sigma"] < 1e-4 * ref


def test_unsupported_paths_and_sizes(mf):
    p, w = _proc(mf, mf.MF_FP64)
    g = p.grid()
    with pytest.raises(mf.MFError):
        p.grad(g, 1, 0, 10)
    with pytest.raises(mf.MFError):
        _proc(mf, mf.MF_FP32_TC)
    with pytest.raises(mf.MFError):
        _proc(mf, mf.MF_FP64, lumi=True)
    edges = torch.tensor(g.get(), dtype=torch.float64, device="cuda").contiguous()
    totals = torch.empty(2 + p.ndim * 50 + 2, dtype=torch.float64, device="cuda")
    with pytest.raises(mf.MFError):
        p.vegas_accumulate_static(edges.view(-1), 50, 1, 0, 0, 10, totals)
    st = _setup(w)
    po = _events(st, 6, 129)
    out = torch.empty(129, dtype=torch.float64, device="cuda")
    p.matrix_element(129, _aos_to_soa(po), out)
    one = torch.empty(1, dtype=torch.float64, device="cuda")
    p.matrix_element(1, _aos_to_soa(po[:1]), one)
    torch.cuda.synchronize()
    assert_fp64_parity(out.cpu().numpy(), st.proc.me2_batched(po), core=1e-13, tail=1e-12, frac=1.0)
    assert one.item() == out[0].item()


@pytest.mark.parametrize("tile", [32, 0])
def test_mixed_with_gluon_processes(mf, tile):
    """e+ e- -> mu+ mu- beside g g -> t t~ and g g -> t t~ g in one mixed
    launch: every process gets its own iteration's result."""
    procs = [_proc(mf, mf.MF_FP64, name=nm)[0] for nm in ("gg_ttx_1tev", "gg_ttxg_13tev", NAME)]
    n = [3000, 1000, 5000]
    mg = [q.grid() for q in procs]
    sg = [q.grid() for q in procs]
    mx = mf.Mixed(procs, mg, n)
    mx.set_launch(0, tile)
    for it in range(2):
        res = mx.run(seed=23, it=it, refine=True)
        for k, q in enumerate(procs):
            ref = q.vegas_iterate(sg[k], 23, it, n[k], refine=True)
            assert res[k]["n_pass"] == ref["n_pass"]
            assert res[k]["I_k"] == pytest.approx(ref["I_k"], rel=1e-12)
            np.testing.assert_allclose(mg[k].get(), sg[k].get(), rtol=0, atol=1e-12)
