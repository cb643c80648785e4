"""The |M|^2 kernel at every launch shape (warps per CTA, CTAs per SM) of the
launch-shape study computes the same events: per-event weights bit for bit
(the same per-warp code), the Vegas sums to summation order, the counters
exactly."""
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


def _run(p, g, n, weights):
    from paper_2211_14056_gb300.sharding import totals_tensor
    p.vegas_accumulate(g, 29, 1, 0, n, weights=weights)
    torch.cuda.synchronize()
    return totals_tensor(g).clone().cpu().numpy()


@pytest.mark.parametrize("precision", [1, 2])
def test_every_launch_shape_gives_the_same_events(mf, precision):
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = WORKLOADS["gg_ttxgg_13tev"]
    p = mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, precision))
    g = p.grid()
    g.set(random_grid(p.ndim, seed=41))
    n = 20011
    ref_w = torch.empty(n, dtype=torch.float64, device="cuda")
    ref = _run(p, g, n, ref_w)
    assert ref[-2] > 0
    for W in range(1, 8):
        cmax = p.set_launch_shape(W)
        assert cmax >= 1
        for c in sorted({1, cmax}):
            p.set_ctas_per_sm(c)
            wt = torch.empty(n, dtype=torch.float64, device="cuda")
            got = _run(p, g, n, wt)
            assert torch.equal(wt, ref_w), (W, c)
            np.testing.assert_array_equal(got[-2:], ref[-2:])
            np.testing.assert_allclose(got[:-2], ref[:-2], rtol=1e-12, atol=0)
    p.set_launch_shape(0)
    p.set_ctas_per_sm(0)


def test_launch_shape_arguments(mf):
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = WORKLOADS["gg_ttxgg_13tev"]
    p64 = mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, mf.MF_FP64))
    with pytest.raises(mf.MFError):
        p64.set_launch_shape(2)
    assert p64.set_launch_shape(0) >= 1
    p32 = mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, mf.MF_FP32))
    with pytest.raises(mf.MFError):
        p32.set_launch_shape(8)
    with pytest.raises(mf.MFError):
        p32.set_launch_shape(-1)
    w3 = WORKLOADS["gg_ttxg_13tev"]
    p3 = mf.Process(PROCESS_IDS[w3["process"]], **process_kwargs(w3, mf.MF_FP32))
    with pytest.raises(mf.MFError):
        p3.set_launch_shape(2)
