"""GPU: checkpoint / resume of a Vegas grid.  The state is the edges and the
recorded iterations (I_k, sigma_k^2); with counter-based random numbers a
grid restored from a checkpoint continues like the original: the same events
and per-event weights, and sums that differ only in their summation order
(the list of events that pass the cuts is built with atomics, so the CTAs'
partial sums add the same weights in a run-dependent order; measured 4e-16
relative on I_k)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14056_gb300 as mf
    return mf


@pytest.mark.parametrize("precision", ["MF_FP64", "MF_FP32"])
def test_resume_from_checkpoint(mf, precision):
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = WORKLOADS["gg_ttxg_13tev"]
    p = mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, getattr(mf, precision)))
    ga = p.grid()
    for it in range(2):
        p.vegas_iterate(ga, seed=11, it=it, n=20000, refine=True)
    state = ga.checkpoint()
    assert state["I_k"].size == 2 and np.all(state["var_k"] > 0)
    ra = p.vegas_iterate(ga, seed=11, it=2, n=20000, refine=True)
    gb = p.grid()
    gb.restore(state)
    rb = p.vegas_iterate(gb, seed=11, it=2, n=20000, refine=True)
    for k in ("n_pass", "iterations"):
        assert ra[k] == rb[k], k
    for k in ("I_k", "sigma_k", "I", "sigma"):
        assert ra[k] == pytest.approx(rb[k], rel=1e-12), k
    assert ra["chi2dof"] == pytest.approx(rb["chi2dof"], rel=1e-9, abs=1e-9)
    np.testing.assert_allclose(ga.get(), gb.get(), rtol=0, atol=1e-13)
    Ia, va = ga.history()
    Ib, vb = gb.history()
    np.testing.assert_array_equal(Ia[:2], Ib[:2])      # the restored record itself is exact
    np.testing.assert_allclose(Ia, Ib, rtol=1e-12)
    np.testing.assert_allclose(va, vb, rtol=1e-9)


def test_history_arguments(mf):
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = WORKLOADS["gg_ttx_1tev"]
    p = mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, mf.MF_FP64))
    g = p.grid()
    assert g.history()[0].size == 0
    with pytest.raises(mf.MFError):
        g.restore({"edges": g.get(), "I_k": np.array([1.0]), "var_k": np.array([0.0])})
    g.restore({"edges": g.get(), "I_k": np.array([1.0, 2.0]), "var_k": np.array([0.5, 0.25])})
    I, v = g.history()
    np.testing.assert_array_equal(I, [1.0, 2.0])
    np.testing.assert_array_equal(v, [0.5, 0.25])


def test_zero_variance_iteration_is_not_recorded(mf):
    """An iteration in which no event passes the cuts (all weights 0, zero
    variance) has no place in the inverse-variance combination: the call
    fails with MF_ERR_ARG and leaves the recorded history as it was, so a
    checkpoint taken afterwards still restores."""
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = dict(WORKLOADS["gg_ttxg_13tev"])
    p = mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, mf.MF_FP64))
    g = p.grid()
    p.vegas_iterate(g, seed=3, it=0, n=4000, refine=False)
    w["pt_cut"] = 1.0e5                        # above sqrt(S) / 2: nothing passes
    q = mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, mf.MF_FP64))
    gq = q.grid()
    gq.restore(g.checkpoint())
    with pytest.raises(mf.MFError) as ei:
        q.vegas_iterate(gq, seed=3, it=1, n=4000, refine=False)
    assert ei.value.status == mf.MF_ERR_ARG
    I, v = gq.history()
    assert I.size == 1 and v[0] > 0
    g2 = p.grid()
    g2.restore(gq.checkpoint())
    r = p.vegas_iterate(g2, seed=3, it=1, n=4000, refine=False)
    assert r["iterations"] == 2
