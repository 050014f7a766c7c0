"""Host-side work split for runs over several GPUs (one process per GPU).

The hologram sum has no exchange step: pixels, and whole problems of a
batch, are independent.  So a multi-GPU run splits problems across ranks
(longest-processing-time-first, by point-pixel updates) and needs no
collective on the data path; only the timing is combined (max over ranks).
"""
from __future__ import annotations

from typing import List, Sequence


def lpt_shard(costs: Sequence[float], world: int) -> List[List[int]]:
    """Partition problem indices over `world` ranks, largest cost first onto
    the least-loaded rank (ties: lowest rank).  Deterministic; every rank
    computes the same answer without communication."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    shards: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        shards[r].append(i)
        load[r] += costs[i]
    return [sorted(s) for s in shards]


def reduce_max(x: float, dist=None, device="cpu") -> float:
    """max over ranks of a host float (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, dist=None, device="cpu") -> float:
    """sum over ranks of a host float (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
