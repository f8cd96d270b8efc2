"""Host logic of the N > 1 benchmark path on CPU: world_size 2 over gloo.
Ranks solve independent problems (no data-path collective); the only
collective is the all-reduce MAX of the timed region."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank               # rank 1 is the slow one
        t, v = bench.aggregate(local_ms, units_per_rank=1e9, steps=4, world=world, dist=dist)
        mine = bench.shard(10, rank, world)
        q.put((rank, t, v, mine, bench.dist_env()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregate_and_shard():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, s0, e0), (r1, t1, v1, s1, e1) = res
    assert t0 == t1 == 15.0                          # max over ranks
    assert v0 == v1 == pytest.approx(2 * 1e9 * 4 / 15e-3)
    assert sorted(s0 + s1) == list(range(10)) and not set(s0) & set(s1)
    assert e0 == (0, 2, 0) and e1 == (1, 2, 1)


def test_single_rank_aggregate_is_identity():
    t, v = bench.aggregate(20.0, 5e9, 2, 1)
    assert t == 20.0 and v == pytest.approx(5e9 * 2 / 20e-3)
