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


def _strip_worker(rank, world, port, q_out, cfg):
    """One y-strip of a periodic grid on this rank: the oracle's boundary pass, then the
    ghost rows replaced by the neighbouring strips' edge rows (one halo exchange per step),
    the x links redone for the corners, and the oracle's step."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from oracle.stepper import WormLBM
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nx, ny, q, steps = cfg["nx"], cfg["ny"], cfg["q"], cfg["steps"]
        h = ny // world
        m = WormLBM(nx, h, q, cfg["mfp"], emulate_3d=True)
        full = np.asarray(cfg["dT"], np.float64)
        m.init_temperature(full[rank * h:(rank + 1) * h])
        up, down = (rank + 1) % world, (rank - 1) % world
        for n in range(1, steps + 1):
            m.apply_bc()
            top = torch.from_numpy(np.ascontiguousarray(m.d[:, h, :]))     # last interior row
            bot = torch.from_numpy(np.ascontiguousarray(m.d[:, 1, :]))     # first interior row
            from_down = torch.empty_like(top)
            from_up = torch.empty_like(bot)
            reqs = [dist.isend(top, up), dist.isend(bot, down),
                    dist.irecv(from_down, down), dist.irecv(from_up, up)]
            for r in reqs:
                r.wait()
            m.d[:, 0, 1:-1] = from_down.numpy()[:, 1:-1]
            m.d[:, h + 1, 1:-1] = from_up.numpy()[:, 1:-1]
            m.d[:, :, 0] = m.d[:, :, nx]                 # x link again: corners from the halos
            m.d[:, :, nx + 1] = m.d[:, :, 1]
            hops, paused = m.sched.advance(n)
            m.d = m.collide_stream(m.d, hops, paused)
            m.n = n
        q_out.put((rank, m.d[:, 1:-1, 1:-1].copy()))
    finally:
        dist.destroy_process_group()


def test_y_strip_decomposition_with_halo_exchange():
    """Spatial decomposition of a periodic grid into y-strips on two gloo ranks: one
    exchanged halo row per step (the planes' edge rows) reproduces the single-domain run
    exactly, so the step needs no other communication."""
    import numpy as np
    import torch.multiprocessing as mp
    from oracle.stepper import WormLBM
    rng = np.random.default_rng(4)
    cfg = dict(nx=14, ny=12, q=16, mfp=3.0, steps=17, dT=rng.standard_normal((12, 14)) * 0.4)
    ref = WormLBM(cfg["nx"], cfg["ny"], cfg["q"], cfg["mfp"], emulate_3d=True)
    ref.init_temperature(cfg["dT"])
    ref.step(cfg["steps"])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_strip_worker, args=(r, 2, port, q, cfg)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([res[0], res[1]], axis=1)
    np.testing.assert_array_equal(got, ref.d[:, 1:-1, 1:-1])


def test_autotune_cache_signature_and_store(tmp_path, monkeypatch):
    """The autotuning cache (host logic, no GPU): the signature ignores the order of the
    grids, separates storage types, shapes and builds of the library, and a stored pick
    is read back; a damaged cache file reads as empty."""
    import torch
    from paper_1911_00180_gb300 import autotune as AT
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "GB300 (test)")
    monkeypatch.setenv("WLBM_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    a = dict(nx=64, ny=16, q=32, bc=(1, 1, 2, 2))
    b = dict(nx=40, ny=40, q=16, bc=(0, 0, 0, 0), mfp_field=object())
    s0 = AT.signature([a, b], 0)
    assert AT.signature([b, a], 0) == s0
    assert AT.signature([a, b], 1) != s0
    assert AT.signature([a, dict(b, q=24)], 0) != s0
    monkeypatch.setattr(AT, "_build_identity", lambda: [1, 2])
    assert AT.signature([a, b], 0) != s0                  # another build of the library
    AT._store("k", {"variant": 3, "graph_steps": 48, "ms_per_step": 0.5})
    assert AT._load()["k"]["graph_steps"] == 48
    (tmp_path / "cache.json").write_text("{not json")
    assert AT._load() == {}
