"""Multi-rank host logic on CPU (gloo, world size 2): ranks take disjoint,
work-balanced shares of the independent instances, every instance is solved
exactly once (here by the oracle, standing in for the GPU), and the timing
reduction takes the max over ranks."""
import os

import numpy as np
import pytest

from paper_2509_03015_gb300 import inputs, sharding


def test_shards_partition_and_balance():
    shapes = inputs.mpc_batch_shapes(K=512)
    for world in (1, 2, 4, 8):
        parts = sharding.shard_instances(shapes, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(512))
        loads = [sum(sharding.instance_work(*shapes[k]) for k in p) for p in parts]
        assert max(loads) <= 1.05 * (sum(loads) / world) + max(sharding.instance_work(*s) for s in shapes)


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    shapes = [(int(N), int(n)) for N, n in inputs.mpc_batch_shapes(K=16, N_hi=64)]
    mine = sharding.rank_share(shapes, rank, world)
    res = {}
    for k in mine:
        N, n = shapes[k]
        s = inputs.kalman_btd(N, n, max(n // 2, 1), 1, 0.95, k)
        res[k] = float(np.abs(oracle.solve_system(s["A_diag"], s["A_sub"], s["B"])).sum())
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    gathered = [None] * world
    dist.all_gather_object(gathered, res)
    if rank == 0:
        merged = {}
        for g in gathered:
            assert not set(g) & set(merged)
            merged.update(g)
        out.put((sorted(merged), float(t.item())))
    dist.destroy_process_group()


def test_two_rank_gloo_shards_cover_batch_once():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    keys, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert keys == list(range(16)) and tmax == 2.0
