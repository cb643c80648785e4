"""The library's side of event sharding, on one GPU.

A rank of a multi-GPU run integrates its own range of the global Philox event
stream (mf_vegas_accumulate with first_event), the ranks' Vegas totals are
summed (the one all-reduce of an iteration), and every rank finishes the
iteration from the summed totals (mf_vegas_finish with the global event
count).  Here the shards run one after the other on one device and the sum is
taken on the device: the result must be that of one mf_vegas_iterate over all
events: the same per-event weights bit for bit, I_k, sigma_k and the refined
grid to 1e-12, the histogram to rounding, and the pass and Newton counters
exactly.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests.inputs import random_grid  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14056_gb300 as mf
    return mf


@pytest.mark.parametrize("name,precision,sizes", [("gg_ttxg_13tev", 0, (1500, 1500)),
                                                  ("gg_ttxgg_13tev", 0, (1000, 2001)),
                                                  ("gg_ttxgg_13tev", 1, (40000, 25536, 7))])
def test_shards_equal_one_iteration(mf, name, precision, sizes):
    from paper_2211_14056_gb300.sharding import totals_tensor
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = WORKLOADS[name]
    p = mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, precision))
    edges = random_grid(p.ndim, seed=23)
    n = sum(sizes)
    seed, it = 13, 2
    ref_grid = p.grid()
    ref_grid.set(edges)
    w_ref = torch.empty(n, dtype=torch.float64, device="cuda")
    ref = p.vegas_iterate(ref_grid, seed, it, n, refine=True, weights=w_ref)
    ref_tot = totals_tensor(ref_grid).clone()
    grids, first = [], 0
    w_sh = torch.empty(n, dtype=torch.float64, device="cuda")
    for m in sizes:
        g = p.grid()
        g.set(edges)
        p.vegas_accumulate(g, seed, it, first, m, weights=w_sh[first:first + m])
        grids.append(g)
        first += m
    summed = totals_tensor(grids[0])
    for g in grids[1:]:
        summed += totals_tensor(g)            # the all-reduce of a multi-rank run
    got_tot = summed.clone()
    r = p.vegas_finish(grids[0], n, refine=True)
    torch.cuda.synchronize()
    assert torch.equal(w_sh, w_ref)
    got, want = got_tot.cpu().numpy(), ref_tot.cpu().numpy()
    np.testing.assert_array_equal(got[-2:], want[-2:])            # passing events, Newton misses
    assert got[-2] == ref["n_pass"] > 0
    np.testing.assert_allclose(got[:-2], want[:-2], rtol=1e-12, atol=0)
    assert r["I_k"] == pytest.approx(ref["I_k"], rel=1e-12)
    assert r["sigma_k"] == pytest.approx(ref["sigma_k"], rel=1e-12)
    assert r["n_pass"] == ref["n_pass"] and r["n_newton_fail"] == ref["n_newton_fail"]
    np.testing.assert_allclose(grids[0].get(), ref_grid.get(), rtol=0, atol=1e-12)


def test_adaptive_helicity_shards_equal_one_iteration(mf):
    """With the adapted helicity draw the totals carry the per-configuration
    sums of squared weights; summed over two shards they refine the table as
    one iteration over all events does (thresholds equal, or a step of 2^-32
    apart where the sums' rounding order differs)."""
    from paper_2211_14056_gb300.sharding import totals_tensor
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = WORKLOADS["gg_ttxgg_13tev"]
    p = mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, 1))
    p.set_helicity_sampling("adaptive")
    edges = random_grid(p.ndim, seed=24)
    sizes = (30000, 20001)
    n = sum(sizes)
    ref_grid = p.grid()
    ref_grid.set(edges)
    w_ref = torch.empty(n, dtype=torch.float64, device="cuda")
    ref = p.vegas_iterate(ref_grid, 14, 1, n, refine=True, weights=w_ref)
    ref_tot = totals_tensor(ref_grid).clone()
    grids, first = [], 0
    w_sh = torch.empty(n, dtype=torch.float64, device="cuda")
    for m in sizes:
        g = p.grid()
        g.set(edges)
        p.vegas_accumulate(g, 14, 1, first, m, weights=w_sh[first:first + m])
        grids.append(g)
        first += m
    summed = totals_tensor(grids[0])
    assert summed.numel() == 2 + p.ndim * grids[0].nbins + 2 + 32
    for g in grids[1:]:
        summed += totals_tensor(g)
    r = p.vegas_finish(grids[0], n, refine=True)
    torch.cuda.synchronize()
    assert torch.equal(w_sh, w_ref)
    np.testing.assert_allclose(summed.cpu().numpy()[-32:], ref_tot.cpu().numpy()[-32:], rtol=1e-12)
    assert r["I_k"] == pytest.approx(ref["I_k"], rel=1e-12)
    assert np.max(np.abs(grids[0].helicity() - ref_grid.helicity())) <= 2.0 ** -32
    assert ref_grid.helicity().max() > 1.5 / 32               # the table did adapt
