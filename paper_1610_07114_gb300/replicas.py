"""Several GPUs, one process each: independent lattices sharded across ranks.

The lattice update has no exchange step between independent lattices, so a batch of
lattices (or a stream of requests) is partitioned across ranks and every rank advances
its share with no collective on the data path.  The only collectives are the barrier
around a timed region and the maximum of the per-rank times (weak scaling: every rank
keeps the same amount of work as ranks are added).  These helpers work on any
torch.distributed backend (NCCL between GPUs; gloo on CPU for tests).
"""
from __future__ import annotations

import heapq
import os


def dist_env():
    """(world, rank, local_rank) from the launcher's environment (1, 0, 0 when absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(work, world: int, rank: int) -> list[int]:
    """Indices of the items rank `rank` of `world` takes: longest item first to the rank
    with the least work so far (ties to the lowest rank).  Every rank computes the same
    assignment from the same list; the shares are disjoint and cover all items, and
    no rank holds more than the mean plus the largest item."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    order = sorted(range(len(work)), key=lambda i: (-work[i], i))
    heap = [(0, r) for r in range(world)]
    mine = []
    for i in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(i)
        heapq.heappush(heap, (load + work[i], r))
    return sorted(mine)


def _device_for(dist):
    import torch

    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def max_over_ranks(x: float, world: int) -> float:
    """Largest value of `x` over all ranks (x itself with one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=_device_for(dist))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=_device_for(dist))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
