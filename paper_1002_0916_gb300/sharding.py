"""Host-side work split for runs over several GPUs (one process per GPU).

The hologram sum (Eq. 1) has no exchange step: pixels, and whole problems
of a batch, are independent.  So a multi-GPU run either splits the rows of
one hologram into slabs, one per rank (each computed with cgh_forward_rows),
or splits the problems of a batch across ranks (longest-processing-time
first, by point-pixel updates), and needs no collective on the data path;
only the timing is combined (max over ranks).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def row_slabs(Ny: int, world: int, align: int = 32) -> List[Tuple[int, int]]:
    """Contiguous slabs (y0, rows) of an Ny-row hologram, one per rank,
    covering every row once: whole groups of `align` rows (the direct
    kernel's tile height) dealt out as evenly as possible, the first ranks
    taking one group more, the ragged last group on the last non-empty
    slab.  A rank may get no rows (rows == 0) when there are fewer groups
    than ranks.  Deterministic; every rank computes the same answer."""
    if world < 1 or Ny < 1 or align < 1:
        raise ValueError("need world >= 1, Ny >= 1, align >= 1")
    groups = (Ny + align - 1) // align
    base, extra = divmod(groups, world)
    out, g0 = [], 0
    for r in range(world):
        ng = base + (1 if r < extra else 0)
        y0 = min(Ny, g0 * align)
        y1 = min(Ny, (g0 + ng) * align)
        out.append((y0, y1 - y0))
        g0 += ng
    return out


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
