"""Multi-rank host logic on CPU (gloo, world size 2): the problem split of a
batch and the max-over-ranks timing that bench.py reports."""
import os
import socket

import pytest

from paper_1002_0916_gb300.sharding import lpt_shard, reduce_max, reduce_sum
from workloads import batch_problems


def test_lpt_shard_partitions_and_balances():
    costs = [c.pp for c in batch_problems(seed=0)]
    for world in (1, 2, 3, 8):
        shards = lpt_shard(costs, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in s) for s in shards]
        # LPT bound: max load <= 4/3 of the optimum (>= mean load)
        assert max(loads) <= (4.0 / 3.0) * (sum(costs) / world) + max(costs)
    assert lpt_shard([5, 1, 1], 2) == [[0], [1, 2]]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [c.pp for c in batch_problems(seed=0)]
        mine = lpt_shard(costs, world)[rank]
        shards = [None] * world
        dist.all_gather_object(shards, mine)
        ms = 10.0 + rank           # each rank's own step time
        pp = float(sum(costs[i] for i in mine))
        q.put((rank, shards, reduce_max(ms, dist), reduce_sum(pp, dist)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    costs = [c.pp for c in batch_problems(seed=0)]
    for rank, shards, mx, total in res:
        assert shards == lpt_shard(costs, 2)          # same split on every rank
        assert mx == 11.0                              # the slowest rank's time
        assert total == pytest.approx(float(sum(costs)))  # whole-job work
    assert sorted(i for s in res[0][1] for i in s) == list(range(len(costs)))


def test_row_slabs_cover_every_row_once():
    from paper_1002_0916_gb300.sharding import row_slabs
    for Ny in (1, 5, 31, 32, 33, 1024, 1080, 2160):
        for world in (1, 2, 3, 4, 8):
            slabs = row_slabs(Ny, world)
            assert len(slabs) == world
            y = 0
            for y0, rows in slabs:
                assert y0 == y and rows >= 0
                assert rows == 0 or y0 % 32 == 0      # whole tile rows
                y += rows
            assert y == Ny
            sizes = [r for _, r in slabs]
            # balanced to one tile row, plus the ragged last group
            assert max(sizes) - min(sizes) <= 64
    assert row_slabs(1024, 2) == [(0, 512), (512, 512)]


def _slab_worker(rank, world, port, q):
    """Each rank computes its own slab of rows with no exchange; the slabs
    are gathered only to check them (the FP64 oracle stands in for the GPU
    method on this CPU-only test)."""
    import numpy as np
    import torch.distributed as dist

    import oracle
    from paper_1002_0916_gb300.sharding import row_slabs
    from workloads import workload
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = workload("cfg1_256x256_n64")
        y0, rows = row_slabs(c.Ny, world)[rank]
        mine = oracle.forward(c, rows=np.arange(y0, y0 + rows, dtype=np.int32))
        parts = [None] * world
        dist.all_gather_object(parts, (y0, mine))
        q.put((rank, parts))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_row_split():
    import numpy as np
    import torch.multiprocessing as mp

    import oracle
    from workloads import workload
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    c = workload("cfg1_256x256_n64")
    whole = oracle.forward(c)
    for rank, parts in res:
        assert [y0 for y0, _ in parts] == [0, 128]
        assert np.array_equal(np.concatenate([m for _, m in parts], 0), whole)
