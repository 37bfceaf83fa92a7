"""N > 1 host logic on CPU with world_size-2 gloo process groups: shell
sharding, timing aggregation, and a failing rank surfacing as an error on the
other rank (no GPU involved)."""
import datetime
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2603_05447_gb300 import dist as gdist


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _init(rank, world, port, timeout_s=30):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=timeout_s))


def _worker_shard(rank, world, port, weights, q):
    _init(rank, world, port)
    mine = gdist.shard(weights, world, rank)
    everyone = [None] * world
    dist.all_gather_object(everyone, mine)
    mx = gdist.max_over_ranks(float(rank + 1))
    sm = gdist.sum_over_ranks(float(sum(weights[i] for i in mine)))
    q.put((rank, everyone, mx, sm))
    dist.destroy_process_group()


def test_shards_cover_each_shell_once_and_timings_combine():
    import random
    rnd = random.Random(4)
    weights = [rnd.randint(100_000, 20_000_000) for _ in range(64)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker_shard, args=(r, 2, port, weights, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, everyone, mx, sm in res:
        flat = sorted(i for part in everyone for i in part)
        assert flat == list(range(64))
        assert mx == 2.0
        assert sm == float(sum(weights))
        loads = [sum(weights[i] for i in part) for part in everyone]
        assert max(loads) <= sum(weights) / 2 + max(weights)


def _worker_fail(rank, world, port, q):
    _init(rank, world, port, timeout_s=5)
    if rank == 1:
        q.put((rank, "raised"))
        raise SystemExit(3)          # a rank that leaves between steps
    try:
        gdist.max_over_ranks(1.0)    # the survivor's next collective must fail, not hang
        q.put((rank, "no error"))
    except Exception as e:           # noqa: BLE001 - any collective error is the detection
        q.put((rank, "error: " + type(e).__name__))


def test_a_lost_rank_surfaces_as_an_error_on_the_survivor():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker_fail, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res[1] == "raised"
    assert res[0].startswith("error")


def test_shard_edge_cases():
    assert gdist.shard([5], 2, 0) == [0] and gdist.shard([5], 2, 1) == []
    assert gdist.shard([], 3, 2) == []
    parts = [gdist.shard([1] * 10, 4, r) for r in range(4)]
    assert sorted(i for p in parts for i in p) == list(range(10))
    assert all(2 <= len(p) <= 3 for p in parts)
