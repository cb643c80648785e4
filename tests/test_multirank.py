"""Event sharding with a totals all-reduce, on two CPU ranks (gloo).

Each rank integrates its own shard of the global Philox event stream with the
oracle, packs the Vegas totals the way the library's totals buffer is laid out
(sum w, sum w^2, histogram, passing events, Newton misses), all-reduces them
with the product's ``allreduce_totals`` and refines.  The result must equal a
single process integrating all events: same I_k, sigma_k and refined grid.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

from oracle import integrate as oi, vegas as ov

CFG = dict(process="gg_ttxg", mt=173.0, wt=0.0, gs=1.2177, sqrt_s=13000.0, lumi=True, pt_cut=30.0, dr_cut=0.0)
N_PER_RANK = 300


def _pack(r):
    return np.concatenate([[r["sum_w"], r["sum_w2"]], r["hist"].ravel(), [np.sum(r["w"] != 0), 0.0]])


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2211_14056_gb300.sharding import allreduce_totals, shard_range
    st = oi.Setup(CFG, amplitude="bg")
    edges = ov.uniform_grid(st.ndim)
    first, n = shard_range(rank, world, N_PER_RANK)
    r = oi.iteration(st, 7, 0, None, edges, events=np.arange(first, first + n))
    tot = torch.tensor(_pack(r), dtype=torch.float64)
    allreduce_totals(tot)
    t = tot.numpy()
    ntot = world * N_PER_RANK
    I, var = ov.estimate(t[0], t[1], ntot)
    hist = t[2:2 + st.ndim * 50].reshape(st.ndim, 50)
    out[rank] = (I, var, ov.refine(edges, hist), t[-2])
    dist.destroy_process_group()


def test_two_rank_sharding_matches_single_process():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    st = oi.Setup(CFG, amplitude="bg")
    edges = ov.uniform_grid(st.ndim)
    ref = oi.iteration(st, 7, 0, 2 * N_PER_RANK, edges)
    ref_edges = ov.refine(edges, ref["hist"])
    for rank in range(2):
        I, var, e, npass = out[rank]
        assert I == pytest.approx(ref["I"], rel=1e-13)
        assert var == pytest.approx(ref["var"], rel=1e-11)
        np.testing.assert_allclose(e, ref_edges, rtol=0, atol=1e-13)
        assert npass == np.sum(ref["w"] != 0)


def test_shard_ranges():
    from paper_2211_14056_gb300.sharding import shard_range
    assert shard_range(0, 4, 10) == (0, 10)
    assert shard_range(3, 4, 10) == (30, 10)
    with pytest.raises(ValueError):
        shard_range(4, 4, 10)
