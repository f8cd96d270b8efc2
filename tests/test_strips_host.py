"""One grid split into row strips over two ranks (gloo, world size 2, CPU):
halo exchange every k layers and an OR all-reduce of the ranks' flags give
the oracle's distances bit for bit. The strips' own work runs through a CPU
stand-in engine (the paper's layer rule on distances)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_2004_00540_gb300 import strips
from strip_cpu_engine import CpuStripEngine


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case(kind):
    if kind == "bernoulli":
        m = synth.bernoulli(90, 70, 0.3, 7)
        return m, synth.sample_free(m, 3, 8)
    m = synth.dfs_maze(61, 45, 9)
    return m, synth.sample_free(m, 1, 10)


def _worker(rank, world, port, kind, k, max_layers, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m, t = _case(kind)
        a, b, ea, eb = strips.strip_rows(m.shape[0], world, rank, k)
        eng = CpuStripEngine(m[ea:eb])
        comm = strips.TorchComm(dist, rank, world)
        a, b, own, L = strips.solve_rank(m, t, world, rank, k, eng, comm, max_layers)
        q.put((rank, a, b, own, L))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind,k,max_layers", [("bernoulli", 4, 0), ("maze", 3, 0), ("maze", 5, 40),
                                               ("bernoulli", 7, 0)])
def test_two_rank_strips_equal_oracle(kind, k, max_layers):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, kind, k, max_layers, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    m, t = _case(kind)
    want, L = oracle.bfs(m, t, max_layers=max_layers)
    got = np.empty_like(want)
    for _, a, b, own, Lr in res:
        got[a:b] = own
        assert Lr == L
    assert res[0][2] == res[1][1]                    # the strips tile the rows
    assert np.array_equal(got, want)


@pytest.mark.parametrize("world,k", [(1, 4), (3, 2), (4, 6)])
def test_local_strips_equal_oracle(world, k):
    """The same rounds with all ranks in one process (the emulation used on
    one GPU), on the CPU engine."""
    m = synth.bernoulli(80, 57, 0.35, 21)
    t = synth.sample_free(m, 2, 22)
    engines = []
    for r in range(world):
        _, _, ea, eb = strips.strip_rows(80, world, r, k)
        engines.append(CpuStripEngine(m[ea:eb]))
    got, L = strips.LocalComms.solve(m, t, world, k, engines)
    want, Lw = oracle.bfs(m, t)
    assert L == Lw and np.array_equal(got, want)


def test_strip_rows_partition_and_errors():
    rows = [strips.strip_rows(103, 4, r, 5) for r in range(4)]
    assert rows[0][0] == 0 and rows[-1][1] == 103
    for (a0, b0, _, _), (a1, b1, _, _) in zip(rows, rows[1:]):
        assert b0 == a1 and b0 - a0 >= 5
    assert rows[1][2] == rows[1][0] - 5 and rows[0][2] == 0 and rows[-1][3] == 103
    with pytest.raises(ValueError):
        strips.strip_rows(9, 2, 0, 5)                # strips shorter than the halo
    with pytest.raises(ValueError):
        strips.strip_rows(100, 2, 2, 5)
