"""Shared helpers of the GPU parity tests: run the CUDA library through its
C ABI and the CPU oracle on the same seeded input, compare bit for bit."""
import numpy as np

import oracle
import paper_2004_00540_gb300 as pkg


def oracle_solve(mask, targets, starts, max_layers=0):
    d, L = oracle.bfs(mask, targets, max_layers)
    off, cells, status = oracle.trace(mask, d, starts)
    return d, L, off, cells, status


def gpu_solve(mask, targets, starts, dist_bits=0, variant=None, depth=None, max_layers=0,
              plain=False, check_every=1):
    with pkg.Planner(mask, dist_bits) as pl:
        if variant is not None:
            pl.set_tuning(variant, depth)
        L = pl.propagate(targets, max_layers, plain=plain, check_every=check_every)
        d = pl.distances()
        paths = pl.trace(starts)
        stats = pl.stats()
    return d, L, paths, stats


def widen(d):
    """uint16 plane -> uint32 with the oracle's sentinel."""
    if d.dtype == np.uint16:
        return np.where(d == 0xFFFF, oracle.INF, d.astype(np.uint32)).astype(np.uint32)
    return d


def assert_parity(mask, targets, starts, **kw):
    max_layers = kw.get("max_layers", 0)
    od, oL, ooff, ocells, ostatus = oracle_solve(mask, targets, starts, max_layers)
    gd, gL, paths, stats = gpu_solve(mask, targets, starts, **kw)
    gd = widen(gd)
    if not np.array_equal(gd, od):
        bad = np.argwhere(gd != od)
        y, x = bad[0]
        raise AssertionError(f"{len(bad)} cells differ; first ({y},{x}) gpu={gd[y, x]} "
                             f"oracle={od[y, x]}; stats={stats}")
    assert gL == oL, (gL, oL)
    assert np.array_equal(paths.status, ostatus)
    assert np.array_equal(paths.offsets, ooff)
    assert np.array_equal(paths.cells, ocells)
    return stats
