"""Batched and continuously batched solving: every grid's distances and paths
are the same bit for bit as the oracle's (and so as the grid solved alone),
whatever else is in the batch, in whatever order and round it arrives."""
import numpy as np
import pytest

import oracle
import synth
import paper_2004_00540_gb300 as pkg
from gpu_util import widen

pytestmark = pytest.mark.gpu


def small_members(n, side_hi=300, base_seed=4):
    return [synth.c4_member(i, base_seed, 64, side_hi) for i in range(n)]


def check(b, tk, w):
    dist, paths, layers = b.result(tk, w.starts.size)
    od, oL = oracle.bfs(w.mask, w.targets)
    assert np.array_equal(widen(dist), od), w.name
    assert layers == oL
    off, cells, status = oracle.trace(w.mask, od, w.starts)
    assert np.array_equal(paths.offsets, off)
    assert np.array_equal(paths.status, status)
    assert np.array_equal(paths.cells, cells)


@pytest.mark.parametrize("per_grid", [False, True])
@pytest.mark.parametrize("shape", [0, 1, 12])
def test_batch_all_at_once(shape, per_grid):
    ws = small_members(24)
    with pkg.Batch(1 << 30, variant=shape) as b:
        b.set_mode(per_grid)
        tks = [b.submit(w.mask, w.targets, w.starts, w.dist_bits) for w in ws]
        assert all(t is not None for t in tks)
        running, done = b.run(0)
        assert running == 0 and done == len(ws)
        for tk, w in zip(tks, ws):
            assert b.poll(tk) == pkg.MPN_BATCH_DONE
            check(b, tk, w)
            b.release(tk)
        assert b.stats()["arena_used"] == 0


@pytest.mark.parametrize("per_grid", [False, True])
def test_batch_wait_runs_rounds_until_done(per_grid):
    ws = small_members(6, side_hi=260, base_seed=60)
    with pkg.Batch(1 << 30) as b:
        b.set_mode(per_grid)
        tks = [b.submit(w.mask, w.targets, w.starts, w.dist_bits) for w in ws]
        # short rounds: the wait takes several of them; the others advance too
        assert b.wait(tks[3], 2) == pkg.MPN_BATCH_DONE
        assert b.stats()["rounds"] > 1
        check(b, tks[3], ws[3])
        for tk, w in zip(tks, ws):
            assert b.wait(tk) == pkg.MPN_BATCH_DONE
            check(b, tk, w)


@pytest.mark.parametrize("per_grid", [False, True])
@pytest.mark.parametrize("shape", [0, 12])
def test_batch_continuous_arrivals_and_short_rounds(shape, per_grid):
    ws = small_members(30, side_hi=400, base_seed=40)
    rng = np.random.default_rng(1)
    order = rng.permutation(len(ws))
    with pkg.Batch(1 << 30, variant=shape) as b:
        b.set_mode(per_grid)
        b.set_depth(16)
        tickets = {}
        pending = list(order)
        rounds = 0
        while pending or any(b.poll(t) == pkg.MPN_BATCH_PENDING for t in tickets):
            for _ in range(int(rng.integers(0, 4))):          # a few arrivals per round
                if pending:
                    i = pending.pop()
                    tickets[b.submit(ws[i].mask, ws[i].targets, ws[i].starts, ws[i].dist_bits)] = i
            b.run(int(rng.integers(1, 6)))                     # short rounds: grids span rounds
            rounds += 1
            assert rounds < 100000
        for tk, i in tickets.items():
            check(b, tk, ws[i])
        assert b.stats()["rounds"] > 3
        assert b.stats()["graph"] == 1          # rounds replayed from a captured CUDA graph


def test_batch_admission_by_memory():
    ws = small_members(12, side_hi=500, base_seed=90)
    with pkg.Batch(3 << 20) as b:                               # room for only a few grids
        admitted, refused = [], []
        for w in ws:
            tk = b.submit(w.mask, w.targets, w.starts, w.dist_bits)
            (admitted if tk is not None else refused).append((tk, w))
        assert admitted and refused
        b.run(0)
        for tk, w in admitted:
            check(b, tk, w)
            b.release(tk)
        # freed memory admits the rest
        for _, w in refused[:3]:
            tk = b.submit(w.mask, w.targets, w.starts, w.dist_bits)
            assert tk is not None
            b.run(0)
            check(b, tk, w)
            b.release(tk)


def test_batch_rejects_bad_endpoints_and_overflow_fails_alone():
    ws = small_members(6, base_seed=7)
    bad = ws[0]
    obst = np.flatnonzero(bad.mask.reshape(-1))[:1].astype(np.uint32)
    with pkg.Batch(1 << 28) as b:
        with pytest.raises(pkg.MPNError) as e:
            b.submit(bad.mask, obst, bad.starts, bad.dist_bits)
        assert e.value.status == pkg.MPN_EOBSTACLE
        with pytest.raises(pkg.MPNError) as e:
            b.submit(bad.mask, bad.targets, np.array([bad.H * bad.W], np.uint32), bad.dist_bits)
        assert e.value.status == pkg.MPN_EINVAL
        corridor = synth.empty(1, 70000)                  # distances past 65534 in uint16
        to = b.submit(corridor, np.array([0], np.uint32), np.array([69999], np.uint32), 16)
        good = [(b.submit(w.mask, w.targets, w.starts, w.dist_bits), w) for w in ws[1:]]
        while b.stats()["running"] or b.stats()["admitted"]:
            b.run(0)
        assert b.poll(to) == pkg.MPN_BATCH_FAILED
        assert b.error(to) == pkg.MPN_EOVERFLOW
        for tk, w in good:
            check(b, tk, w)


@pytest.mark.parametrize("per_grid", [False, True])
def test_batch_fixed_depth(per_grid):
    w = synth.c4_member(2, 4, 64, 300)
    with pkg.Batch(1 << 28) as b:
        b.set_mode(per_grid)
        tk = b.submit(w.mask, w.targets, w.starts, w.dist_bits, max_layers=9)
        b.run(0)
        dist, paths, layers = b.result(tk, w.starts.size)
    od, oL = oracle.bfs(w.mask, w.targets, max_layers=9)
    assert np.array_equal(widen(dist), od) and layers == oL


@pytest.mark.parametrize("per_grid", [False, True])
def test_batch_full_size_members_sample(per_grid):
    ws = [synth.c4_member(i) for i in (0, 1, 2, 3, 101, 254, 255)]
    with pkg.Batch(16 << 30) as b:
        b.set_mode(per_grid)
        tks = [b.submit(w.mask, w.targets, w.starts, w.dist_bits) for w in ws]
        b.run(0)
        for tk, w in zip(tks, ws):
            check(b, tk, w)


@pytest.mark.parametrize("per_grid", [False, True])
def test_serve_on_the_real_engine_matches_oracle_alone_and_in_the_mix(per_grid):
    """The continuous-batching loop (serve) on the real batched engine:
    Poisson arrivals, rounds of a few sweeps so that requests arriving while
    others are on the GPU join later rounds, every served path kept. Each
    response equals the oracle's paths for that grid, i.e. the result of the
    grid solved alone, whatever else was in flight."""
    from paper_2004_00540_gb300.serve import Request, serve
    ws = small_members(20, side_hi=360, base_seed=120)
    arr = synth.poisson_arrivals(len(ws), 400.0, seed=3)
    reqs = [Request(w.mask, w.targets, w.starts, w.dist_bits, float(a)) for w, a in zip(ws, arr)]
    with pkg.Batch(1 << 30) as b:
        b.set_mode(per_grid)
        rep = serve(b, reqs, round_sweeps=4, keep_results=True, max_round_sweeps=16)
        assert b.stats()["graph"] == 1
    assert not rep.failed and len(rep.results) == len(ws)
    assert rep.rounds > 3
    for i, w in enumerate(ws):
        od, _ = oracle.bfs(w.mask, w.targets)
        off, cells, status = oracle.trace(w.mask, od, w.starts)
        got = rep.results[i]
        assert np.array_equal(got.offsets, off), w.name
        assert np.array_equal(got.status, status), w.name
        assert np.array_equal(got.cells, cells), w.name
    # one grid served alone gives the same response
    with pkg.Batch(1 << 28) as b:
        alone = serve(b, [Request(ws[5].mask, ws[5].targets, ws[5].starts, ws[5].dist_bits, 0.0)],
                      round_sweeps=4, keep_results=True)
    assert np.array_equal(alone.results[0].cells, rep.results[5].cells)
    assert np.array_equal(alone.results[0].offsets, rep.results[5].offsets)


def test_batch_without_lookahead_same_results(monkeypatch):
    """Blocks that only wait at a sweep's end (lookahead off, a test hook)
    give the same paths as the default, where they run ready tiles of the
    next sweep meanwhile; both equal the oracle's."""
    ws = small_members(10, side_hi=420, base_seed=150)
    monkeypatch.setenv("MPN_TEST_NO_LOOKAHEAD", "1")
    with pkg.Batch(1 << 30) as b:
        b.set_mode(False)             # the lookahead is the global-sweep mode's
        tks = [b.submit(w.mask, w.targets, w.starts, w.dist_bits) for w in ws]
        b.run(3)                      # a short round, then the rest
        b.run(0)
        for tk, w in zip(tks, ws):
            check(b, tk, w)


def test_batch_long_walks_in_segments():
    """Grids whose walks are far longer than the rest (serpentine corridors,
    both dtypes) in one batch with ordinary grids: their long walks go in
    segments found with a jump table; every path equals the oracle's."""
    def serp(H, W):
        m = np.ones((H, W), np.uint8)
        m[0::2, :] = 0
        for r in range(1, H, 2):
            m[r, W - 1 if (r // 2) % 2 == 0 else 0] = 0
        return m
    ws = small_members(6, side_hi=300, base_seed=170)
    extra = []
    for H, W, bits in ((121, 401, 16), (161, 511, 32)):
        m = serp(H, W)
        free = np.flatnonzero(m.reshape(-1) == 0)
        st = np.concatenate([[free[-1], free[len(free) // 3], 3], free[::997]]).astype(np.uint32)
        extra.append(synth.Workload(f"serp{H}x{W}", m, np.array([0], np.uint32), st, bits, {}))
    with pkg.Batch(1 << 30) as b:
        tks = [(b.submit(w.mask, w.targets, w.starts, w.dist_bits), w) for w in ws + extra]
        b.run(0)
        for tk, w in tks:
            check(b, tk, w)


def test_batch_mode_only_while_empty():
    w = synth.c4_member(2, 4, 64, 300)
    with pkg.Batch(1 << 28) as b:
        b.set_mode(True)
        tk = b.submit(w.mask, w.targets, w.starts, w.dist_bits)
        with pytest.raises(pkg.MPNError):
            b.set_mode(False)                    # a grid is in the batch
        b.run(0)
        check(b, tk, w)
        b.release(tk)
        b.set_mode(False)                        # empty again
        tk = b.submit(w.mask, w.targets, w.starts, w.dist_bits)
        b.run(0)
        check(b, tk, w)
