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
