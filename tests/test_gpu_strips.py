"""The resume call (mpn_propagate_resume) and one grid split into row strips
run on the library, with the ranks emulated round by round on one GPU; both
against the CPU oracle, bit for bit."""
import numpy as np
import pytest

import oracle
import synth
import paper_2004_00540_gb300 as pkg
from paper_2004_00540_gb300 import strips
from gpu_util import widen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bits", [16, 32])
def test_resume_from_oracle_prefix_equals_full_solve(bits):
    """Cells of the oracle's plane up to layer f kept, the rest (whatever the
    plane holds there) recomputed: the result is the full solve, from a host
    and from a device plane, to convergence and to a fixed layer."""
    torch = pytest.importorskip("torch")
    m = synth.bernoulli(300, 257, 0.3, 31)
    t = synth.sample_free(m, 3, 32)
    d, L = oracle.bfs(m, t)
    dt = np.uint16 if bits == 16 else np.uint32
    for f in (0, 1, L // 3, L - 1):
        plane = np.where(d <= f, d, np.uint32(12345)).astype(np.uint32)   # junk past f
        plane = np.where(d == oracle.INF, 0xFFFFFFFF, plane).astype(np.uint32)
        host = np.where(plane == 0xFFFFFFFF, 0xFFFF, plane).astype(np.uint16) if bits == 16 else plane
        with pkg.Planner(m, bits) as pl:
            got_L = pkg.mpn_propagate_resume(pl.ctx, host, f)
            assert got_L == (L if L > f else 0)
            assert np.array_equal(widen(pl.distances()), d)
            dev = torch.from_numpy(host.view(np.int16 if bits == 16 else np.int32)).cuda()
            cap = f + 3
            pkg.mpn_propagate_resume(pl.ctx, dev, f, cap)
            want, _ = oracle.bfs(m, t, max_layers=cap)
            assert np.array_equal(widen(pl.distances()), want)
            # paths traced after a resumed run follow the resumed plane
            st = synth.sample_free(m, 10, 33)
            paths = pl.trace(st)
            off, cells, status = oracle.trace(m, want, st)
            assert np.array_equal(paths.cells, cells) and np.array_equal(paths.status, status)
    with pkg.Planner(m, bits) as pl:
        with pytest.raises(pkg.MPNError):
            pkg.mpn_propagate_resume(pl.ctx, host, 5, 5)        # cap not past the start layer
        bad = np.full(m.shape, 0, dt)                            # obstacles marked reached
        with pytest.raises(pkg.MPNError):
            pkg.mpn_propagate_resume(pl.ctx, bad, 0)


@pytest.mark.parametrize("world,k", [(2, 8), (3, 5), (4, 16)])
def test_strips_on_one_gpu_equal_oracle(world, k):
    m = synth.dfs_maze(257, 301, 41)
    t = synth.sample_free(m, 2, 42)
    engines = [strips.gpu_engine(m, world, r, k) for r in range(world)]
    got, L = strips.LocalComms.solve(m, t, world, k, engines)
    want, Lw = oracle.bfs(m, t)
    assert L == Lw and np.array_equal(got, want)
    m2 = synth.bernoulli(400, 390, 0.25, 43)
    t2 = synth.sample_free(m2, 5, 44)
    engines = [strips.gpu_engine(m2, world, r, k) for r in range(world)]
    got, L = strips.LocalComms.solve(m2, t2, world, k, engines, max_layers=61)
    want, Lw = oracle.bfs(m2, t2, max_layers=61)
    assert L == Lw and np.array_equal(got, want)


def test_invariant_check_accepts_solves_and_flags_a_bad_plane(monkeypatch):
    """mpn_check (the on-device invariant check) finds nothing wrong in solved
    planes (a maze, a Bernoulli grid, a fixed depth, the MPN_CHECK=1 mode of
    mpn_propagate), and counts the cells of a plane that is not a distance map:
    one resumed from a prefix in which two neighbouring cells are 4 apart."""
    torch = pytest.importorskip("torch")
    maze = synth.dfs_maze(301, 257, 51)
    m2 = synth.bernoulli(200, 333, 0.3, 52)
    for m, n in ((maze, 2), (m2, 4)):
        t = synth.sample_free(m, n, 53)
        with pkg.Planner(m, pkg.MPN_DIST_U32) as pl:
            pl.propagate(t)
            assert pkg.mpn_check(pl.ctx) == 0
            pl.propagate(t, max_layers=7)
            assert pkg.mpn_check(pl.ctx) == 0
        monkeypatch.setenv("MPN_CHECK", "1")
        with pkg.Planner(m, pkg.MPN_DIST_U32) as pl:
            assert pl.propagate(t) == oracle.bfs(m, t)[1]
        monkeypatch.delenv("MPN_CHECK")
    e = synth.empty(40, 50)
    plane = np.full((40, 50), 0xFFFFFFFF, np.uint32)
    plane[0, 0] = 0
    plane[0, 2] = 5                  # no cell at 4 next to it: not a distance map
    with pkg.Planner(e, pkg.MPN_DIST_U32) as pl:
        pkg.mpn_propagate_resume(pl.ctx, plane, 5)
        assert pkg.mpn_check(pl.ctx) > 0
        st = pkg.load().mpn_check(pl.ctx, None)
        assert st == pkg.MPN_ECHECK
