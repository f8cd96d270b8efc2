"""CUDA path vs the CPU oracle, bit for bit: distance planes, layer counts,
path offsets, cells and per-start status, on seeded inputs that span many
tiles with ragged edges, every compiled tile shape and several temporal
depths, both distance dtypes, and the five named workloads."""
import numpy as np
import pytest

import oracle
import synth
import paper_2004_00540_gb300 as pkg
from gpu_util import assert_parity, gpu_solve, widen

pytestmark = pytest.mark.gpu


def n_variants():
    n = 0
    while pkg.mpn_variant_info(n) is not None:
        n += 1
    return n


def max_depth(variant):
    return min(32, pkg.mpn_variant_info(variant)["region_rows"] // 3)


def rand_case(H, W, p, nt, ns, seed):
    m = synth.bernoulli(H, W, p, seed) if p > 0 else synth.empty(H, W)
    nfree = int((m == 0).sum())
    if nfree == 0:
        m.reshape(-1)[0] = 0
        nfree = 1
    t = synth.sample_free(m, min(nt, nfree), seed + 1)
    s = np.random.default_rng(seed).integers(0, H * W, size=ns).astype(np.uint32)
    return m, t, s


@pytest.mark.parametrize("H,W", [(1, 1), (1, 77), (93, 1), (2, 2), (37, 1000), (300, 301),
                                 (777, 513), (1000, 1000), (257, 4099)])
@pytest.mark.parametrize("p", [0.0, 0.3])
def test_random_grids_default_tiling(H, W, p):
    m, t, s = rand_case(H, W, p, 3, 60, H * 7919 + W)
    assert_parity(m, t, s)


@pytest.mark.parametrize("variant", range(n_variants()))
@pytest.mark.parametrize("depth", [1, 5, 16, 24, 32])
def test_every_variant_and_depth(variant, depth):
    if depth > max_depth(variant):
        with pkg.Planner(synth.empty(10, 10)) as pl:
            with pytest.raises(pkg.MPNError):
                pl.set_tuning(variant, depth)      # interior shorter than the halo
        return
    m, t, s = rand_case(611, 1403, 0.3, 4, 80, 17 + variant * 40 + depth)
    assert_parity(m, t, s, variant=variant, depth=depth)


@pytest.mark.parametrize("variant", range(n_variants()))
def test_empty_grid_corner_source(variant):
    # worst case for sweeps: one source in a corner of an empty grid
    H, W = 900, 1300
    m = synth.empty(H, W)
    s = np.array([H * W - 1, (H - 1) * W, W - 1, 450 * W + 650], np.uint32)
    stats = assert_parity(m, np.array([0], np.uint32), s, variant=variant,
                          depth=max_depth(variant))
    assert stats["layers"] == max(H, W) - 1


@pytest.mark.parametrize("bits", [16, 32])
def test_dtypes(bits):
    m, t, s = rand_case(200, 250, 0.25, 2, 40, 5)
    d, L, paths, stats = gpu_solve(m, t, s, dist_bits=bits)
    assert d.dtype == (np.uint16 if bits == 16 else np.uint32)
    assert stats["dist_bits"] == bits
    assert_parity(m, t, s, dist_bits=bits)


def test_u16_overflow_reported():
    # a corridor longer than 65534 steps cannot fit a uint16 plane
    m = synth.empty(1, 70000)
    with pkg.Planner(m, pkg.MPN_DIST_U16) as pl:
        with pytest.raises(pkg.MPNError) as e:
            pl.propagate(np.array([0], np.uint32))
        assert e.value.status == pkg.MPN_EOVERFLOW


@pytest.mark.parametrize("L", [1, 2, 7, 40, 1000])
def test_fixed_depth_network(L):
    m, t, s = rand_case(400, 380, 0.3, 2, 50, 99)
    assert_parity(m, t, s, max_layers=L)
    assert_parity(m, t, s, max_layers=L, variant=2, depth=13)


@pytest.mark.parametrize("check_every", [1, 16])
def test_plain_per_layer_kernel(check_every):
    m, t, s = rand_case(300, 333, 0.3, 3, 40, 3)
    assert_parity(m, t, s, plain=True, check_every=check_every)
    w = synth.c1_small()
    assert_parity(w.mask, w.targets, w.starts, plain=True)
    assert_parity(m, t, s, plain=True, max_layers=25)


def test_activity_map_matches_literal_recurrence():
    for seed in range(4):
        m, t, _ = rand_case(40 + seed, 57, 0.3, 1 + seed, 1, 300 + seed)
        with pkg.Planner(m) as pl:
            layers = pl.propagate(t)
            for L in (1, 3, layers, layers + 5):
                got = pl.activity(L)
                assert np.array_equal(got, oracle.omap(m, t, L)), L
            assert np.array_equal(pl.activity(0), oracle.omap(m, t, layers))


def test_errors_and_states():
    m = synth.bernoulli(50, 60, 0.3, 1)
    obst = int(np.flatnonzero(m.reshape(-1))[0])
    free = int(np.flatnonzero(m.reshape(-1) == 0)[0])
    with pkg.Planner(m) as pl:
        with pytest.raises(pkg.MPNError) as e:
            pl.trace(np.array([free], np.uint32))
        assert e.value.status == pkg.MPN_ESTATE
        with pytest.raises(pkg.MPNError) as e:
            pl.propagate(np.array([obst], np.uint32))
        assert e.value.status == pkg.MPN_EOBSTACLE
        with pytest.raises(pkg.MPNError) as e:
            pl.propagate(np.array([50 * 60], np.uint32))
        assert e.value.status == pkg.MPN_EINVAL
        with pytest.raises(pkg.MPNError) as e:
            pl.propagate(np.array([], np.uint32))
        assert e.value.status == pkg.MPN_EINVAL
        pl.propagate(np.array([free], np.uint32))
        with pytest.raises(pkg.MPNError) as e:
            pl.trace(np.array([50 * 60 + 5], np.uint32))
        assert e.value.status == pkg.MPN_EINVAL
        # too small an output: offsets still filled, status ENOMEM
        st = np.array([free, 50 * 60 - 1, obst], np.uint32)
        off = np.zeros(4, np.uint64)
        cells = np.zeros(1, np.uint32)
        status = np.zeros(3, np.int8)
        r = pkg.mpn_trace(pl.ctx, st, off, cells, 0, status)
        d = pl.distances()
        want_total = 1 + (0 if d.reshape(-1)[50 * 60 - 1] == 0xFFFF or m.reshape(-1)[-1]
                          else int(d.reshape(-1)[50 * 60 - 1]) + 1)
        assert r == pkg.MPN_ENOMEM and int(off[-1]) == want_total
        assert status[2] == pkg.MPN_PATH_ON_OBSTACLE
        # empty start list is fine
        p = pl.trace(np.array([], np.uint32))
        assert p.offsets.tolist() == [0]


def test_device_tensors_in_and_out():
    torch = pytest.importorskip("torch")
    m, t, s = rand_case(513, 700, 0.3, 3, 30, 12)
    dm = torch.from_numpy(m).cuda()
    dt = torch.from_numpy(t.astype(np.int32)).cuda()
    ds = torch.from_numpy(s.astype(np.int32)).cuda()
    stream = torch.cuda.current_stream()
    ctx = pkg.mpn_create(dm, 513, 700, 32, stream)
    try:
        L = pkg.mpn_propagate(ctx, dt)
        dd = torch.empty((513, 700), dtype=torch.int32, device="cuda")
        pkg.mpn_get_distances(ctx, dd)
        off = torch.zeros(31, dtype=torch.int64, device="cuda")
        pkg.mpn_trace_lengths(ctx, ds, off)
        total = int(off[-1].item())
        cells = torch.zeros(max(total, 1), dtype=torch.int32, device="cuda")
        status = torch.zeros(30, dtype=torch.int8, device="cuda")
        assert pkg.mpn_trace(ctx, ds, off, cells, total, status) == pkg.MPN_OK
        torch.cuda.synchronize()
    finally:
        pkg.mpn_destroy(ctx)
    od, oL = oracle.bfs(m, t)
    assert L == oL
    assert np.array_equal(dd.cpu().numpy().view(np.uint32), od)
    ooff, ocells, ostatus = oracle.trace(m, od, s)
    assert np.array_equal(off.cpu().numpy().view(np.uint64), ooff)
    assert np.array_equal(cells.cpu().numpy().view(np.uint32)[:total], ocells)
    assert np.array_equal(status.cpu().numpy(), ostatus)


@pytest.mark.parametrize("shift", [0, 1, 4])
def test_page_locked_host_outputs(shift):
    """Results read into page-locked host memory (stored by the GPU over the
    host link), at 16-, 4- and 1-byte alignment, equal the oracle's and those
    read into pageable memory."""
    torch = pytest.importorskip("torch")
    m, t, s = rand_case(613, 900, 0.3, 5, 300, 77)
    n = s.size
    with pkg.Planner(m, 32) as pl:
        pl.propagate(t)
        off_p = pl.trace(s).offsets              # pageable numpy buffers
        total = int(off_p[-1])
        ctx = pl.ctx

        def pinned(nbytes):
            return torch.zeros(nbytes + 16, dtype=torch.uint8).pin_memory()[shift:shift + nbytes]

        hs = torch.from_numpy(s.astype(np.int32)).pin_memory()
        off_b, cells_b, st_b = pinned(8 * (n + 1)), pinned(4 * max(total, 1)), pinned(n)
        assert pkg.mpn_trace(ctx, hs, off_b, cells_b, total, st_b) == pkg.MPN_OK
        len_b = pinned(8 * (n + 1))
        pkg.mpn_trace_lengths(ctx, hs, len_b)
        tgt_b, dist_b = pinned(4 * n), pinned(4 * n)
        pkg.mpn_nearest_targets(ctx, hs, tgt_b, dist_b)
        got_t, got_d = pl.nearest_targets(s)
    d, _ = oracle.bfs(m, t)
    ooff, ocells, ostatus = oracle.trace(m, d, s)
    off = off_b.numpy().copy().view(np.uint64)
    assert np.array_equal(off, ooff) and np.array_equal(off_p, ooff)
    assert np.array_equal(len_b.numpy().copy().view(np.uint64), ooff)
    assert np.array_equal(cells_b.numpy().copy().view(np.uint32)[:total], ocells)
    assert np.array_equal(st_b.numpy().copy().view(np.int8), ostatus)
    assert np.array_equal(tgt_b.numpy().copy().view(np.uint32), got_t)
    assert np.array_equal(dist_b.numpy().copy().view(np.uint32), got_d)


def test_async_distance_copy_is_ordered_before_the_next_propagate():
    """mpn_get_distances_async on a side stream, then at once a propagate from
    other targets on the same context: the copy holds the first plane (the
    propagate waits for it on the device), and the second plane is right."""
    torch = pytest.importorskip("torch")
    m, t, _ = rand_case(1500, 1300, 0.3, 4, 1, 91)
    t2 = synth.sample_free(m, 2, 92)
    side = torch.cuda.Stream()
    h1 = torch.empty((1500, 1300), dtype=torch.int32).pin_memory()
    h2 = torch.empty((1500, 1300), dtype=torch.int32).pin_memory()
    with pkg.Planner(m, 32) as pl:
        pl.propagate(t)
        pkg.mpn_get_distances_async(pl.ctx, h1, side)
        pkg.mpn_propagate(pl.ctx, t2.astype(np.uint32), 0, wait=False)
        pkg.mpn_get_distances_async(pl.ctx, h2)
        pkg.mpn_sync(pl.ctx)
        side.synchronize()
    d1, _ = oracle.bfs(m, t)
    d2, _ = oracle.bfs(m, t2)
    assert np.array_equal(h1.numpy().view(np.uint32), d1)
    assert np.array_equal(h2.numpy().view(np.uint32), d2)


@pytest.mark.parametrize("offset", [0, 1, 8])
def test_device_mask_at_any_alignment(offset):
    """The encoder's vector path needs a 16-byte-aligned mask; a mask at any
    other address takes the byte path. Both give the oracle's plane."""
    torch = pytest.importorskip("torch")
    m, t, s = rand_case(301, 517, 0.3, 3, 5, 70 + offset)
    big = torch.zeros(301 * 517 + 64, dtype=torch.uint8, device="cuda")
    big[offset:offset + 301 * 517] = torch.from_numpy(m.reshape(-1)).cuda()
    dm = big[offset:offset + 301 * 517]
    ctx = pkg.mpn_create(dm, 301, 517, 32, torch.cuda.current_stream())
    try:
        L = pkg.mpn_propagate(ctx, t)
        d = np.empty((301, 517), np.uint32)
        pkg.mpn_get_distances(ctx, d)
    finally:
        pkg.mpn_destroy(ctx)
    od, oL = oracle.bfs(m, t)
    assert L == oL and np.array_equal(d, od)


def test_packed_input_and_set_mask():
    m, t, s = rand_case(130, 200, 0.3, 2, 20, 8)
    P = 8
    bits = np.zeros((130, P), np.uint32)
    free = (m == 0)
    for x in range(200):
        bits[:, x // 32] |= (free[:, x].astype(np.uint32) << np.uint32(x % 32))
    bits[:, 7] = 0xFFFFFFFF                      # junk past the row must be ignored
    ctx = pkg.mpn_create_packed(bits, 130, 200, P, 32)
    try:
        L = pkg.mpn_propagate(ctx, t)
        d = np.empty((130, 200), np.uint32)
        pkg.mpn_get_distances(ctx, d)
    finally:
        pkg.mpn_destroy(ctx)
    od, oL = oracle.bfs(m, t)
    assert L == oL and np.array_equal(d, od)
    m2, t2, s2 = rand_case(130, 200, 0.2, 2, 20, 9)
    with pkg.Planner(m) as pl:
        pl.propagate(t)
        pkg.mpn_set_mask(pl.ctx, m2)
        with pytest.raises(pkg.MPNError):
            pl.distances()                        # new mask invalidates distances
        pl.propagate(t2)
        assert np.array_equal(widen(pl.distances()), oracle.bfs(m2, t2)[0])


def test_workload_c1_small():
    w = synth.c1_small()
    assert_parity(w.mask, w.targets, w.starts, dist_bits=16)


def test_workload_c2_maze():
    w = synth.c2_maze()
    stats = assert_parity(w.mask, w.targets, w.starts)
    assert stats["layers"] > 1000


def test_workload_c3_maze_open():
    w = synth.c3_maze_open()
    assert_parity(w.mask, w.targets, w.starts)


@pytest.mark.parametrize("i", [0, 1, 2, 3, 10, 11, 100, 101, 254, 255])
def test_workload_c4_members(i):
    w = synth.c4_member(i)
    assert_parity(w.mask, w.targets, w.starts, dist_bits=w.dist_bits)


@pytest.mark.parametrize("tiling", [None, (12, 28), (0, 24)])
def test_workload_c5_huge_full(tiling):
    """The full 23170^2 grid: automatic tiling (shape 12, depth 28, the
    tiling the benchmark times after autotuning), the same explicitly, and
    shape 0 at depth 24."""
    w = synth.c5_huge()
    kw = {} if tiling is None else {"variant": tiling[0], "depth": tiling[1]}
    stats = assert_parity(w.mask, w.targets, w.starts, **kw)
    if tiling is None:
        assert (stats["variant"], stats["depth"]) == (12, 28)
    assert stats["layers"] > 100
    # the activation log carried the distances (one entry per word and
    # visit that reached cells in it), and visits stopped early where stable
    assert stats["log_entries"] > 0
    assert stats["tile_visits"] <= stats["tile_layers"] <= stats["tile_visits"] * stats["depth"]


def test_activation_log_counts_match_the_oracle():
    """Every entry is one (word, sweep) pair in which the word gained cells:
    with one visit per tile and sweep, their number is the count of distinct
    (32-cell word, sweep of k layers) pairs among the cells the oracle
    reaches at distance >= 1."""
    m, t, s = rand_case(700, 900, 0.28, 5, 10, 91)
    with pkg.Planner(m) as pl:
        pl.set_tuning(0, 16)
        pl.propagate(t)
        st = pl.stats()
    d, _ = oracle.bfs(m, t)
    H, W = d.shape
    ys, xs = np.nonzero((d != oracle.INF) & (d >= 1))
    sweep = (d[ys, xs].astype(np.int64) - 1) // 16
    pairs = np.unique((ys.astype(np.int64) * ((W + 31) // 32) + xs // 32) * 100000 + sweep)
    assert st["log_entries"] == pairs.size


@pytest.mark.parametrize("chunks,slots", [("0", ""), ("1", ""), ("3", ""), ("", "1"), ("2", "2")])
def test_log_fallbacks_stay_exact(chunks, slots, monkeypatch):
    """The activation log's fallback paths, forced through test hooks: no log
    (the plane is filled and every block writes its distances), a pool of a
    few chunks (most blocks write directly; the decode keeps their cells), and
    a decode that takes only the first visits of a tile from its slots and the
    rest from the header chain. Distances and layer counts equal the oracle's
    on a maze (many visits per tile) and a Bernoulli grid, both dtypes."""
    if chunks:
        monkeypatch.setenv("MPN_TEST_LOG_CHUNKS", chunks)
    if slots:
        monkeypatch.setenv("MPN_TEST_DECODE_SLOTS", slots)
    maze = synth.dfs_maze(512, 512, 62)
    cases = [rand_case(700, 900, 0.3, 5, 1, 61)[:2], (maze, synth.sample_free(maze, 3, 62))]
    for m, t in cases:
        d, L = oracle.bfs(m, t)
        for bits in (16, 32):
            if bits == 16 and L > 65534:
                continue
            with pkg.Planner(m, bits) as pl:
                pl.set_tuning(0, 16)
                assert pl.propagate(t) == L
                got = pl.distances()
            assert np.array_equal(widen(got), d)


@pytest.mark.parametrize("hook,value", [("MPN_TEST_SWEEP_CAP", "2"), ("MPN_TEST_SPIN_LIMIT", "1")])
def test_device_waits_run_out_then_context_recovers(hook, value, monkeypatch):
    """A device-side limit made to run out on purpose: the sweep cap (2
    sweeps on a grid that needs hundreds) or the grid barrier's spin limit (a
    wait of one poll while another block is still in its first visit). The
    kernel records the error and every block returns -- nothing hangs or
    faults -- and the call reports MPN_ETIMEOUT. The same context then solves
    the grid exactly once the hook is gone."""
    m, t, s = rand_case(2048, 2048, 0.3, 1, 20, 91)
    d, L = oracle.bfs(m, t)
    assert L > 200
    with pkg.Planner(m, pkg.MPN_DIST_U32) as pl:
        pl.set_tuning(0, 16)
        monkeypatch.setenv(hook, value)
        with pytest.raises(pkg.MPNError) as e:
            pl.propagate(t)
        assert e.value.status == pkg.MPN_ETIMEOUT
        monkeypatch.delenv(hook)
        assert pl.propagate(t) == L
        assert np.array_equal(widen(pl.distances()), d)
        paths = pl.trace(s)
    off, cells, status = oracle.trace(m, d, s)
    assert np.array_equal(paths.offsets, off) and np.array_equal(paths.status, status)
    assert np.array_equal(paths.cells, cells)


@pytest.mark.parametrize("lookahead", ["0", "1"])
def test_lookahead_on_and_off_equal_oracle(lookahead, monkeypatch):
    """Blocks waiting at the end of a sweep either only wait (hook "1") or run
    tiles of the next sweep whose neighbourhood has finished (default): the
    same distances and paths, equal to the oracle's, on a maze (few tiles per
    sweep) and a Bernoulli grid (many), at two depths and a fixed layer cap."""
    monkeypatch.setenv("MPN_TEST_NO_LOOKAHEAD", "1" if lookahead == "0" else "0")
    maze = synth.dfs_maze(700, 900, 163)
    cases = [rand_case(1500, 1300, 0.3, 4, 30, 161), (maze, synth.sample_free(maze, 2, 164),
                                                       synth.sample_free(maze, 30, 165))]
    for m, t, s in cases:
        for depth in (8, 24):
            with pkg.Planner(m, pkg.MPN_DIST_U32) as pl:
                pl.set_tuning(0, depth)
                d, L = oracle.bfs(m, t)
                assert pl.propagate(t) == L
                assert np.array_equal(widen(pl.distances()), d)
                paths = pl.trace(s)
                off, cells, status = oracle.trace(m, d, s)
                assert np.array_equal(paths.cells, cells) and np.array_equal(paths.offsets, off)
                dL, _ = oracle.bfs(m, t, max_layers=L // 3 + 1)
                pl.propagate(t, max_layers=L // 3 + 1)
                assert np.array_equal(widen(pl.distances()), dL)


def serpentine(H, W):
    """Corridors along every other row, joined at alternating ends: the walk
    from one end to the other is about H * W / 2 steps long."""
    m = np.ones((H, W), np.uint8)
    m[0::2, :] = 0
    for r in range(1, H, 2):
        m[r, W - 1 if (r // 2) % 2 == 0 else 0] = 0
    return m


@pytest.mark.parametrize("bits", [16, 32])
def test_long_walks_split_into_segments_equal_oracle(bits):
    """Walks longer than the split threshold are cut into segments found with
    the jump table and walked side by side; with short walks, unreachable
    starts and starts on obstacles in the same call, every path equals the
    oracle's cell for cell (both dtypes)."""
    m = serpentine(121, 401)
    H, W = m.shape
    free = np.flatnonzero(m.reshape(-1) == 0)
    t = np.array([0], np.uint32)
    rng = np.random.default_rng(5)
    s = np.concatenate([[free[-1], free[-2], free[len(free) // 2], 1 * W + 3, free[5]],
                        rng.choice(free, 40, replace=False)]).astype(np.uint32)
    d, L = oracle.bfs(m, t)
    assert L > 20000
    with pkg.Planner(m, bits) as pl:
        assert pl.propagate(t) == L
        paths = pl.trace(s)
    off, cells, status = oracle.trace(m, d, s)
    assert np.array_equal(paths.status, status) and np.array_equal(paths.offsets, off)
    assert np.array_equal(paths.cells, cells)


def test_autotune_records_choice_and_stays_exact():
    m, t, s = rand_case(1500, 1400, 0.3, 6, 40, 77)
    with pkg.Planner(m) as pl:
        v, d, ms = pl.autotune(t)
        assert 0 <= v < n_variants() and 1 <= d <= max_depth(v) and ms > 0
        st = pl.stats()
        assert (st["variant"], st["depth"]) == (v, d)
        pl.propagate(t)
        assert np.array_equal(widen(pl.distances()), oracle.bfs(m, t)[0])
    # a later context of the same size bucket starts from the measured choice
    m2, t2, s2 = rand_case(1700, 1300, 0.25, 3, 40, 78)
    with pkg.Planner(m2) as pl:
        st = pl.stats()
        assert (st["variant"], st["depth"]) == (v, d)
    assert_parity(m2, t2, s2)


@pytest.mark.parametrize("case", ["empty", "bernoulli", "maze", "c1", "c3"])
def test_euclid_trace_matches_oracle(case):
    if case == "empty":
        m = synth.empty(300, 500)
        t = np.array([0, 299 * 500 + 499], np.uint32)
        s = np.random.default_rng(0).integers(0, 300 * 500, 200).astype(np.uint32)
    elif case == "bernoulli":
        m, t, s = rand_case(700, 900, 0.3, 3, 300, 31)
    elif case == "maze":
        m = synth.dfs_maze(301, 257, 5)
        t = synth.sample_free(m, 2, 6)
        s = np.random.default_rng(1).integers(0, 301 * 257, 100).astype(np.uint32)
    elif case == "c1":
        w = synth.c1_small()
        m, t, s = w.mask, w.targets, w.starts
    else:
        w = synth.c3_maze_open()
        m, t, s = w.mask, w.targets, w.starts
    d, _ = oracle.bfs(m, t)
    ooff, ocells, ostatus = oracle.euclid_trace(m, d, s)
    with pkg.Planner(m) as pl:
        pl.propagate(t)
        p = pl.trace_euclid(s)
    assert np.array_equal(p.status, ostatus)
    assert np.array_equal(p.offsets, ooff)
    assert np.array_equal(p.cells, ocells)


@pytest.mark.parametrize("case", ["bernoulli", "c3"])
def test_nearest_targets(case):
    if case == "bernoulli":
        m, t, s = rand_case(600, 800, 0.3, 12, 500, 41)
    else:
        w = synth.c3_maze_open()
        m, t, s = w.mask, w.targets, w.starts
    d, _ = oracle.bfs(m, t)
    off, cells, status = oracle.trace(m, d, s)
    with pkg.Planner(m) as pl:
        pl.propagate(t)
        got_t, got_d = pl.nearest_targets(s)
    tset = set(int(x) for x in t)
    for i in range(s.size):
        if status[i] != 0:
            assert got_t[i] == 0xFFFFFFFF and got_d[i] == 0xFFFFFFFF
            continue
        assert got_t[i] == cells[off[i + 1] - 1] and int(got_t[i]) in tset
        assert got_d[i] == d.reshape(-1)[s[i]]
    # the reached target is a nearest one: its own BFS distance to the start
    # equals the start's multi-source distance
    for i in np.flatnonzero(status == 0)[:20]:
        dt, _ = oracle.bfs(m, [int(got_t[i])])
        assert dt.reshape(-1)[s[i]] == d.reshape(-1)[s[i]]
