"""The allocation-free accumulation entry point (mf_vegas_accumulate_static).

Host programs that hand out all device memory themselves cannot let this
library call cudaMalloc; for them the fused kernel's scratch is a fixed array
inside the library.  Its output must equal that of mf_vegas_accumulate, the
entry point whose scratch comes from mf_grid_create, on two calls in a row
(the second call reuses the array the first one left behind).  The two entry
points run different kernels: the static one the fused sample + |M|^2 +
accumulate kernel (k_fused), the other the two-kernel path (sampling records,
then |M|^2 and accumulation), which the parity tests hold to the oracle; this
comparison is what pins the fused kernel.  Kept in its own file, collected
last, so a failure here stops a -x run only after every other test has run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


class _View:
    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": "<f8", "data": (ptr, False),
                                         "version": 3, "strides": None}


@pytest.mark.parametrize("name,precision,nbins", [("gg_ttxgg_13tev", 1, 50), ("gg_ttxg_13tev", 0, 50),
                                                 ("gg_ttx_1tev", 0, 64)])
def test_static_scratch_matches_grid_scratch(name, precision, nbins):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14056_gb300 as mf
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = WORKLOADS[name]
    p = mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, precision))
    g = p.grid(nbins)
    edges = torch.tensor(g.get(), dtype=torch.float64, device="cuda").contiguous()
    ptr, cnt = g.totals()
    n = 50000
    for call, (seed, it) in enumerate([(11, 0), (12, 3)]):
        totals = torch.full((cnt,), float("nan"), dtype=torch.float64, device="cuda")
        w_static = torch.empty(n, dtype=torch.float64, device="cuda")
        w_grid = torch.empty(n, dtype=torch.float64, device="cuda")
        p.vegas_accumulate_static(edges, g.nbins, seed, it, 1000 * call, n, totals, weights=w_static)
        p.vegas_accumulate(g, seed, it, 1000 * call, n, weights=w_grid)
        torch.cuda.synchronize()
        ref = torch.as_tensor(_View(ptr, cnt), device="cuda").clone()
        got, ref = totals.cpu().numpy(), ref.cpu().numpy()
        # per-event weights: the fused kernel and the two-kernel path on the
        # same events (the same per-event arithmetic in both)
        assert torch.equal(w_static, w_grid)
        # sums and histogram: equal up to the order of in-CTA atomics
        np.testing.assert_allclose(got[:-2], ref[:-2], rtol=1e-12, atol=0)
        np.testing.assert_array_equal(got[-2:], ref[-2:])
        assert got[-2] > 0
