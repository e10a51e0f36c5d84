"""Multi-process host logic on CPU (gloo, world size 2): work sharding and the
slowest-rank timing used by the benchmark under torchrun."""
import os
import socket

import pytest

from paper_1911_00180_gb300 import dist as D


def test_shard_partitions_items():
    for n in (0, 1, 5, 96, 97):
        for world in (1, 2, 3, 8):
            got = sorted(i for r in range(world) for i in D.shard(n, r, world))
            assert got == list(range(n))
            sizes = [len(D.shard(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def test_shard_by_cost_balances_and_partitions():
    costs = [float((k * 37) % 11 + 1) for k in range(40)]
    for world in (2, 3, 4):
        parts = [D.shard_by_cost(costs, r, world) for r in range(world)]
        assert sorted(i for p in parts for i in p) == list(range(40))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = D.shard(96, rank, world)
        q.put((rank, mine, D.max_over_ranks(10.0 + rank), D.sum_over_ranks(len(mine))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_shares_and_slowest_time():
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
    res.sort()
    assert sorted(res[0][1] + res[1][1]) == list(range(96))
    assert res[0][2] == res[1][2] == 11.0
    assert res[0][3] == res[1][3] == 96.0
