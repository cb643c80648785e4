"""Event sharding across ranks (one process per GPU).

Events are independent (arXiv:2211.14056, abstract: the generator is
"parallelized in the event axis"), and the Philox counter is the global event
index, so rank r of a world of size W integrates events [r*n, (r+1)*n) of the
same stream.  The only exchange is one sum of the Vegas totals per iteration
(sum w, sum w^2, the per-bin sums of w^2 and two counters: 2 + 50 d + 2
doubles); every rank then refines its grid identically.
"""


def shard_range(rank, world, n_per_rank):
    """(first global event, count) of this rank's shard (weak scaling)."""
    if not (0 <= rank < world) or n_per_rank < 1:
        raise ValueError("bad shard")
    return rank * n_per_rank, n_per_rank


class _CudaArray:
    """__cuda_array_interface__ view of a library-owned device buffer."""

    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": "<f8", "data": (ptr, False),
                                         "version": 3, "strides": None}


def totals_tensor(grid):
    """The grid's device totals as a torch tensor aliasing the library buffer."""
    import torch
    ptr, cnt = grid.totals()
    return torch.as_tensor(_CudaArray(ptr, cnt), device="cuda")


def allreduce_totals(totals, group=None):
    """Sum a totals tensor over all ranks in place (NCCL for CUDA tensors, gloo for CPU)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(totals, group=group)
    return totals
