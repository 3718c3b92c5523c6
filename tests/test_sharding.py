"""Multi-rank host logic on CPU: world-size-2 gloo process groups."""
import os
import socket

import numpy as np
import pytest

from paper_1902_03252_gb300 import sharding, workloads as W


def test_balanced_shards_cover_and_balance():
    w = W.c3(batch=64)
    work = [g.nodes * w.n_pot for g in w.grids]
    for world in (1, 2, 3, 8):
        sh = sharding.balanced_shards(work, world)
        flat = sorted(i for s in sh for i in s)
        assert flat == list(range(64))
        loads = [sum(work[i] for i in s) for s in sh]
        assert max(loads) - min(loads) <= max(work)
        assert sh == sharding.balanced_shards(work, world)  # deterministic


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.c3(batch=16)
    work = [g.nodes * w.n_pot for g in w.grids]
    mine = sharding.shard_for(work, rank, world)
    # every rank sees the same partition; gather the shards to check coverage
    out = [None] * world
    dist.all_gather_object(out, mine)
    t = sharding.reduce_max(float(rank + 1) * 1.5)
    # per-sample placeholder results (10 x sample index + 0.5), computed only
    # by the rank that owns the sample, gathered back in sample order
    vals = [10.0 * i + 0.5 for i in mine]
    full = sharding.gather_in_order(vals, mine, len(work))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out, t, full))


def test_two_rank_gloo_sharding_and_max():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, out, t, full in res:
        assert t == 3.0  # max over ranks of (rank + 1) * 1.5
        flat = sorted(i for s in out for i in s)
        assert flat == list(range(16))
        assert not (set(out[0]) & set(out[1]))
        assert out[0] and out[1]  # both ranks own samples
        assert full == [10.0 * i + 0.5 for i in range(16)]  # every rank, sample order


def test_gather_in_order_single_process_and_errors():
    with pytest.raises(ValueError):
        sharding.gather_in_order([1.0], [0], 2)            # sample 1 in no shard
    with pytest.raises(ValueError):
        sharding.gather_in_order([1.0, 2.0], [0, 0], 1)    # sample 0 twice
    assert sharding.gather_in_order([2.0, 1.0], [1, 0], 2) == [1.0, 2.0]
