"""One graph counted by several GPUs, one process per GPU.

The CSR is replicated, every rank computes the levels and the cover edges
(they are the same on every rank: the BFS levels are unique given the root
rule), counts one work-balanced slice of the edge index space through
``tc_count_range``, and the slice counts are summed by one all-reduce of a
single 64-bit integer.  The count is a sum of independent per-edge terms
over the cover edges (Alg. 1, Thm. 2 of Bader et al., "Triangle Counting
Through Cover-Edges"), so the sum over any partition is the total.
"""
from __future__ import annotations


def count_sharded(graph, mode: int, rank: int, world_size: int, all_reduce) -> tuple[int, int]:
    """Count this rank's slice of ``graph`` and sum over the ranks.

    ``graph`` exposes ``shard_bounds(mode, nshards)`` and
    ``count_range(mode, begin, end)`` (``paper_2210_00389_gb300.Graph``
    does); ``all_reduce(int) -> int`` sums one integer over the ranks.
    Returns (this rank's count, the total).
    """
    if not 0 <= rank < world_size:
        raise ValueError(f"rank {rank} not in [0, {world_size})")
    bounds = graph.shard_bounds(mode, world_size)
    if len(bounds) != world_size + 1 or bounds[0] != 0 or any(
            bounds[k] > bounds[k + 1] for k in range(world_size)):
        raise RuntimeError(f"invalid shard bounds {list(bounds)}")
    local = int(graph.count_range(mode, int(bounds[rank]), int(bounds[rank + 1])))
    return local, int(all_reduce(local))


def torch_all_reduce_sum(device=None, group=None):
    """An ``all_reduce`` for count_sharded over torch.distributed (NCCL on
    GPUs, gloo on CPU): counts are below 2^63, so one int64 carries them."""
    import torch
    import torch.distributed as dist

    def reduce(value: int) -> int:
        t = torch.tensor([value], dtype=torch.int64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return int(t.item())

    return reduce
