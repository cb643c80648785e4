"""GPU: the mixed launch (several processes in one sampling launch and one
persistent |M|^2 launch) gives each process the same iteration as its own
mf_vegas_iterate; CUDA-graph replay and the autotuner leave results intact."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

NAMES = ["gg_ttx_1tev", "gg_ttxg_13tev", "gg_ttxgg_13tev"]


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14056_gb300 as mf
    return mf


def _procs(mf, precision):
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    return [mf.Process(PROCESS_IDS[WORKLOADS[k]["process"]], **process_kwargs(WORKLOADS[k], precision))
            for k in NAMES]


@pytest.mark.parametrize("precision,tile", [(0, 32), (1, 32), (2, 32), (0, 0), (1, 0)])
def test_mixed_matches_separate_iterations(mf, precision, tile):
    # FP64: identical up to summation order, over two refined iterations.
    # FP32: the two kernels inline the amplitude code differently (FMA
    # contraction), so events agree to FP32 rounding; after a refinement the
    # grids differ at that level and single events can cross a cut, so FP32 is
    # compared on one iteration of the uniform grid.
    tol = 1e-12 if precision == 0 else 1e-6
    iters = 2 if precision == 0 else 1
    procs = _procs(mf, precision)
    n = [6000, 3000, 1500]
    mixed_grids = [p.grid() for p in procs]
    solo_grids = [p.grid() for p in procs]
    mx = mf.Mixed(procs, mixed_grids, n)
    mx.set_launch(0, tile)                       # tile 0: each process's own |M|^2 kernel
    for it in range(iters):
        res = mx.run(seed=21, it=it, refine=True)
        for k, p in enumerate(procs):
            ref = p.vegas_iterate(solo_grids[k], 21, it, n[k], refine=True)
            assert res[k]["n_pass"] == ref["n_pass"]
            assert res[k]["I_k"] == pytest.approx(ref["I_k"], rel=tol)
            assert res[k]["sigma_k"] == pytest.approx(ref["sigma_k"], rel=100 * tol)
            np.testing.assert_allclose(mixed_grids[k].get(), solo_grids[k].get(), rtol=0, atol=tol)
    assert res[2]["iterations"] == iters


def test_mixed_graph_replay_and_autotune(mf):
    procs = _procs(mf, 1)
    n = [20000, 8000, 3000]
    ga = [p.grid() for p in procs]
    gb = [p.grid() for p in procs]
    plain = mf.Mixed(procs, ga, n)
    graph = mf.Mixed(procs, gb, n)
    graph.use_graph(True)
    side = torch.cuda.Stream()                   # capture needs a non-default stream
    cands = [(1, 8), (2, 8), (1, 32), (2, 32), (0, 0)]
    times, best = graph.autotune(seed=5, candidates=cands, stream=side)
    assert len(times) == 5 and 0 <= best < 5 and all(t > 0 for t in times)
    plain.set_launch(*cands[best])
    for it in range(3):
        a = plain.run(seed=5, it=it, refine=True)
        b = graph.run(seed=5, it=it, refine=True, stream=side)
        for k in range(3):
            assert a[k]["n_pass"] == b[k]["n_pass"]
            # same kernels, same launch shape: per-event results identical, sums up to atomics order
            assert a[k]["I_k"] == pytest.approx(b[k]["I_k"], rel=1e-12)
            assert b[k]["iterations"] == it + 1
            np.testing.assert_allclose(ga[k].get(), gb[k].get(), rtol=0, atol=1e-12)


def test_mixed_rejects_bad_plans(mf):
    procs = _procs(mf, 1)
    p64 = _procs(mf, 0)
    g = [p.grid() for p in procs]
    with pytest.raises(mf.MFError):
        mf.Mixed([procs[0], p64[1]], [g[0], p64[1].grid()], [10, 10])     # mixed precision
    with pytest.raises(mf.MFError):
        mf.Mixed([procs[0]], [g[1]], [10])                                 # grid of another process
    with pytest.raises(mf.MFError):
        mf.Mixed(procs, g, [10, 1, 10])                                    # too few events
    plan = mf.Mixed(procs, g, [10, 10, 10])
    with pytest.raises(mf.MFError):
        plan.set_launch(0, -1)                                             # negative tile
    with pytest.raises(mf.MFError):
        plan.autotune(seed=1, candidates=[(1, 8), (-1, 8)])                # negative CTAs per SM
