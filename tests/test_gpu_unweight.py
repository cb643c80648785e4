"""GPU: hit-or-miss unweighting (mf_unweight) against the oracle.

The GPU evaluates the events as in an iteration and keeps event e if
r_e w_max < w_e, r_e from the second Philox stream.  Against the oracle's
weights, its uniforms of that stream and oracle.unweight:
  * the set of kept events is the oracle's (the order of the output is not
    fixed, its set is); an event whose decision is within the weights'
    FP64 parity of the threshold would be ambiguous, and none is expected;
  * kept weights (1, or w / w_max for overweight events), their momenta and
    the counts of kept and overweight events;
  * a full output buffer: MF_WARN_CAPACITY, the total still counted, the
    written events a subset of the kept ones;
  * FP32 weights give the FP64 decisions except where the FP32 weight lies on
    the other side of the threshold; the estimate w_max * sum(weights) / n
    agrees with the iteration's I_k within its statistical error;
  * with helicity sampling on, the weights unweighted are the sampled ones:
    the kept set is the oracle's for its sampled weights.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import integrate as oi, philox as oph, unweight as ou, vegas as ov  # noqa: E402
from tests.inputs import random_grid  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14056_gb300 as mf
    return mf


def _proc(mf, name, precision):
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = WORKLOADS[name]
    return mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, precision)), w


def _run(p, g, seed, it, first, n, w_max, cap):
    mom = torch.full((p.n_ext * 4 * max(cap, 1),), float("nan"), dtype=torch.float64, device="cuda")
    wt = torch.full((max(cap, 1),), float("nan"), dtype=torch.float64, device="cuda")
    ev = torch.full((max(cap, 1),), -1, dtype=torch.int64, device="cuda")
    kept, over, st = p.unweight(g, seed, it, first, n, w_max, cap, mom, wt, ev)
    torch.cuda.synchronize()
    m = min(kept, cap)
    return (kept, over, st, ev[:m].cpu().numpy(), wt[:m].cpu().numpy(),
            mom.view(p.n_ext, 4, max(cap, 1))[:, :, :m].permute(2, 0, 1).cpu().numpy())


@pytest.mark.parametrize("name,n,amp", [("gg_ttxg_13tev", 20000, "bg"), ("uux_ttxgg_13tev", 3000, "feynman")])
def test_unweighting_matches_oracle(mf, name, n, amp):
    from paper_2211_14056_gb300.workloads import oracle_cfg
    p, w = _proc(mf, name, mf.MF_FP64)
    g = p.grid()
    edges = random_grid(p.ndim, seed=29)
    g.set(edges)
    seed, it, first = 37, 4, 1000
    st = oi.Setup(oracle_cfg(w), amplitude=amp)
    events = np.arange(first, first + n, dtype=np.uint64)
    y = oph.uniforms(seed, it, events, st.ndim)
    wo, _ = st.weights(y, edges)
    r = oph.unweight_uniforms(seed, it, events)
    w_max = 0.4 * wo.max()                      # some events overweight
    kept_o, weight_o = ou.unweight(wo, r, w_max)
    # decisions within the FP64 parity of the threshold would be ambiguous
    ambiguous = np.abs(r * w_max - wo) <= 1e-10 * np.abs(wo)
    assert not np.any(ambiguous & (wo > 0))
    kept, over, status, ev, wt, mom = _run(p, g, seed, it, first, n, w_max, n)
    assert status == mf.MF_OK
    assert kept == int(kept_o.sum()) > 0 and over == int((kept_o & (wo > w_max)).sum()) > 0
    order = np.argsort(ev)
    ev, wt, mom = ev[order], wt[order], mom[order]
    idx = np.flatnonzero(kept_o)
    np.testing.assert_array_equal(ev, events[idx].astype(np.int64))
    np.testing.assert_allclose(wt, weight_o[idx], rtol=1e-10)
    assert np.all(wt[wo[idx] <= w_max] == 1.0)
    po = st.kinematics(y[:, idx], edges)[0]
    scale = 2 * po[:, 0, 0][:, None, None]
    assert np.max(np.abs(mom - po) / scale) < 1e-12
    # the grid records nothing
    assert g.history()[0].size == 0


def test_capacity_and_fp32(mf):
    name, n, seed, it = "gg_ttxgg_13tev", 30000, 5, 0
    p64, w = _proc(mf, name, mf.MF_FP64)
    p32, _ = _proc(mf, name, mf.MF_FP32)
    edges = random_grid(p64.ndim, seed=30)
    g64, g32 = p64.grid(), p32.grid()
    g64.set(edges)
    g32.set(edges)
    wt = torch.empty(n, dtype=torch.float64, device="cuda")
    r64 = p64.vegas_iterate(g64, seed, it, n, refine=False, weights=wt)
    w64 = wt.cpu().numpy()
    w_max = 5.0 * w64[w64 > 0].mean()          # ~10% of the events kept, some overweight
    g64.reset()
    k64, o64, st, ev64, wt64, _ = _run(p64, g64, seed, it, 0, n, w_max, n)
    assert st == mf.MF_OK and k64 > 100
    # the estimate: w_max * sum of kept weights / n against I_k
    est = w_max * wt64.sum() / n
    x = np.zeros(n)
    x[ev64] = w_max * wt64
    assert abs(est - r64["I_k"]) < 5 * x.std() / np.sqrt(n)
    # a buffer for half of them
    cap = k64 // 2
    k, o, st, ev, wt_half, _ = _run(p64, g64, seed, it, 0, n, w_max, cap)
    assert st == mf.MF_WARN_CAPACITY and k == k64 and o == o64 and ev.size == cap
    assert np.all(np.isin(ev, ev64)) and np.unique(ev).size == cap
    # FP32 weights: the same decisions except across the threshold
    k32, _, _, ev32, _, _ = _run(p32, g32, seed, it, 0, n, w_max, n)
    r = oph.unweight_uniforms(seed, it, np.arange(n, dtype=np.uint64))
    wt32 = torch.empty(n, dtype=torch.float64, device="cuda")
    p32.vegas_iterate(g32, seed, it, n, refine=False, weights=wt32)
    w32 = wt32.cpu().numpy()
    differ = np.setxor1d(ev64, ev32)
    assert np.all((r[differ] * w_max < w32[differ]) != (r[differ] * w_max < w64[differ]))
    print(f"FP32 vs FP64 unweighting: {differ.size} of {k64} decisions differ (weights across the threshold)")
    assert differ.size <= max(2, k64 // 1000)


def test_arguments(mf):
    p, _ = _proc(mf, "gg_ttx_1tev", mf.MF_FP64)
    g = p.grid()
    with pytest.raises(mf.MFError):
        p.unweight(g, 1, 0, 0, 100, 0.0, 0)
    with pytest.raises(mf.MFError):
        p.unweight(g, 1, 0, 0, 0, 1.0, 0)
    k, o, st = p.unweight(g, 1, 0, 0, 1000, 1e-30, 0)          # nothing written, all counted
    assert st == mf.MF_WARN_CAPACITY and k > 0


def test_unweighting_with_helicity_sampling(mf):
    from paper_2211_14056_gb300.workloads import oracle_cfg
    from oracle import helicity as oh
    p, w = _proc(mf, "gg_ttxg_13tev", mf.MF_FP64)
    p.set_helicity_sampling(True)
    g = p.grid()
    edges = random_grid(p.ndim, seed=37)
    g.set(edges)
    seed, it, first, n = 38, 2, 500, 8000
    st = oi.Setup(oracle_cfg(w), amplitude="bg")
    events = np.arange(first, first + n, dtype=np.uint64)
    y = oph.uniforms(seed, it, events, st.ndim)
    wo, _, _ = oh.sampled_weights(st, y, edges, seed, it, events)
    r = oph.unweight_uniforms(seed, it, events)
    w_max = 0.4 * wo.max()
    kept_o, weight_o = ou.unweight(wo, r, w_max)
    ambiguous = np.abs(r * w_max - wo) <= 1e-10 * np.abs(wo)
    assert not np.any(ambiguous & (wo > 0))
    kept, over, status, ev, wt, mom = _run(p, g, seed, it, first, n, w_max, n)
    assert status == mf.MF_OK and kept == int(kept_o.sum()) > 0
    order = np.argsort(ev)
    np.testing.assert_array_equal(ev[order], events[np.flatnonzero(kept_o)].astype(np.int64))
    np.testing.assert_allclose(wt[order], weight_o[kept_o], rtol=1e-10)
