"""The N > 1 host path on CPU: two gloo ranks shard a batch of independent
problems (disjoint, complete, balanced) and reduce their timing scalars."""
import os
import socket

import pytest

from paper_1706_06844_gb300 import shard


def test_shard_is_a_balanced_partition():
    costs = [shard.problem_cost(n, n) for n in [63, 511, 127, 255, 511, 63, 255, 127, 511]]
    for world in (1, 2, 3, 4):
        parts = [shard.shard(costs, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)
    with pytest.raises(ValueError):
        shard.shard(costs, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, costs, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard.shard(costs, rank, world)
        # each rank "times" its own share; the job time is the maximum
        t = shard.max_over_ranks(sum(costs[i] for i in mine), dist)
        units = shard.sum_over_ranks(len(mine), dist)
        out.put((rank, mine, t, units))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    costs = [shard.problem_cost(n, n) for n in [63, 127, 255, 511] * 5]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, t0, u0), (r1, m1, t1, u1) = res
    assert sorted(m0 + m1) == list(range(len(costs))) and not set(m0) & set(m1)
    assert t0 == t1 == max(sum(costs[i] for i in m0), sum(costs[i] for i in m1))
    assert u0 == u1 == len(costs)
