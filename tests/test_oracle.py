"""Pins for the CPU oracle against what the paper and mathematics fix:
hand-worked layer maps, brute-force shortest paths, closed forms on empty
grids, exhaustive tiny grids, and path invariants. None of these re-types the
oracle's own code."""
import heapq
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
INF = oracle.INF
NB8 = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]


def dijkstra(mask, targets):
    """Textbook Dijkstra with a binary heap, unit weights on 8 moves."""
    H, W = mask.shape
    dist = np.full((H, W), INF, np.int64)
    pq = []
    for t in targets:
        y, x = divmod(int(t), W)
        dist[y, x] = 0
        heapq.heappush(pq, (0, y, x))
    while pq:
        d, y, x = heapq.heappop(pq)
        if d > dist[y, x]:
            continue
        for dy, dx in NB8:
            ny, nx = y + dy, x + dx
            if 0 <= ny < H and 0 <= nx < W and not mask[ny, nx] and d + 1 < dist[ny, nx]:
                dist[ny, nx] = d + 1
                heapq.heappush(pq, (d + 1, ny, nx))
    return dist


def _read_golden_omap():
    blocks, cur, name = {}, None, None
    for line in open(os.path.join(GOLD, "omap_5x5_layers.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line == "mask" or line.startswith("layer"):
            name = line
            blocks[name] = []
            continue
        blocks[name].append(line.split())
    return blocks


def test_golden_hand_worked_layers():
    b = _read_golden_omap()
    rows = b["mask"]
    mask = np.array([[1 if c == "#" else 0 for c in r] for r in rows], np.uint8)
    src = [y * 5 + x for y, r in enumerate(rows) for x, c in enumerate(r) if c == "S"]
    for L in (1, 2, 3):
        want = np.array(b[f"layer {L}"], np.int64)
        got = oracle.omap(mask, src, L)
        assert np.array_equal(got, want), (L, got)


def test_paper_layer_statements():
    # after layer 1: source = 2, its free neighbours = 1; source = n + 1 after
    # layer n; obstacles stay 0 (Methods, "Activity Map Generation")
    m = synth.bernoulli(21, 23, 0.25, 4)
    m[10, 11] = 0
    src = [10 * 23 + 11]
    A1 = oracle.omap(m, src, 1)
    assert A1[10, 11] == 2
    for dy, dx in NB8:
        assert A1[10 + dy, 11 + dx] == (0 if m[10 + dy, 11 + dx] else 1)
    for n in range(1, 30):
        A = oracle.omap(m, src, n)
        assert A[10, 11] == n + 1
        assert not A[m != 0].any()


@pytest.mark.parametrize("seed", range(12))
def test_bfs_equals_literal_recurrence(seed):
    # O_L = max(0, L + 1 - d) for every L up to past convergence
    H, W = 9 + seed, 13 + 2 * seed
    m = synth.bernoulli(H, W, 0.3, 1000 + seed)
    free = np.flatnonzero(m.reshape(-1) == 0)
    rng = np.random.default_rng(seed)
    tg = rng.choice(free, size=1 + seed % 3, replace=False)
    d, layers = oracle.bfs(m, tg)
    di = d.astype(np.int64)
    for L in range(0, layers + 3):
        A = oracle.omap(m, tg, L).astype(np.int64)
        want = np.where(di != INF, np.maximum(0, L + 1 - di), 0)
        assert np.array_equal(A, want), L
        assert np.array_equal(oracle.distance_from_activity(A, L),
                              np.where(di <= L, di, INF).astype(np.uint32))


@pytest.mark.parametrize("seed", range(200))
def test_bfs_vs_dijkstra_random_tiny(seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(1, 17)), int(rng.integers(1, 17))
    m = (rng.random((H, W)) < rng.uniform(0, 0.6)).astype(np.uint8)
    free = np.flatnonzero(m.reshape(-1) == 0)
    if free.size == 0:
        return
    tg = rng.choice(free, size=int(rng.integers(1, min(4, free.size) + 1)), replace=False)
    d, layers = oracle.bfs(m, tg)
    ref = dijkstra(m, tg)
    assert np.array_equal(d.astype(np.int64), ref)
    fin = ref[ref != INF]
    assert layers == int(fin.max())


def test_exhaustive_4x4_all_masks_all_targets():
    # all 2^16 obstacle masks of a 4 x 4 grid, every free single target:
    # compare with all-pairs shortest paths by Floyd-Warshall (batched numpy)
    n = 16
    masks = ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    big = 99
    D = np.full((1 << n, n, n), big, np.int16)
    for c in range(n):
        D[:, c, c] = 0
        cy, cx = divmod(c, 4)
        for dy, dx in NB8:
            y, x = cy + dy, cx + dx
            if 0 <= y < 4 and 0 <= x < 4:
                e = y * 4 + x
                ok = (masks[:, c] == 0) & (masks[:, e] == 0)
                D[ok, c, e] = 1
    for k in range(n):
        D = np.minimum(D, D[:, :, k:k + 1] + D[:, k:k + 1, :])
    bad = 0
    for mi in range(1 << n):
        m = masks[mi].reshape(4, 4)
        for t in np.flatnonzero(masks[mi] == 0):
            d, _ = oracle.bfs(m, [t])
            want = D[mi, t].astype(np.int64)
            want = np.where((want >= big) | (masks[mi] != 0), INF, want)
            bad += not np.array_equal(d.reshape(-1).astype(np.int64), want)
    assert bad == 0


@pytest.mark.parametrize("H,W,k", [(1, 1, 1), (1, 50, 2), (37, 1, 1), (64, 64, 3), (1500, 1100, 7)])
def test_chebyshev_closed_form_empty_grid(H, W, k):
    rng = np.random.default_rng(H * W + k)
    tg = rng.choice(H * W, size=k, replace=False)
    d, layers = oracle.bfs(np.zeros((H, W), np.uint8), tg)
    yy, xx = np.mgrid[0:H, 0:W]
    want = np.full((H, W), np.iinfo(np.int64).max, np.int64)
    for t in tg:
        ty, tx = divmod(int(t), W)
        want = np.minimum(want, np.maximum(np.abs(yy - ty), np.abs(xx - tx)))
    assert np.array_equal(d.astype(np.int64), want)
    assert layers == int(want.max())


@pytest.mark.parametrize("n", [5, 9, 101, 1001])
def test_centre_and_corner_longest_path(n):
    # empty square, source in the middle: longest path 0.5 n (odd n: (n-1)/2);
    # corner source is the worst case, n - 1 (Results, run-time sections)
    z = np.zeros((n, n), np.uint8)
    c = (n // 2) * n + n // 2
    assert oracle.bfs(z, [c])[1] == (n - 1) // 2
    assert oracle.bfs(z, [0])[1] == n - 1
    assert oracle.bfs(z, [(n - 1) * n])[1] == n - 1


def test_more_sources_never_increase_distance():
    m = synth.bernoulli(120, 90, 0.3, 8)
    free = np.flatnonzero(m.reshape(-1) == 0)
    rng = np.random.default_rng(0)
    order = rng.permutation(free)[:12]
    prev = None
    prev_layers = None
    for k in range(1, 13):
        d, layers = oracle.bfs(m, order[:k])
        if prev is not None:
            assert (d <= prev).all()
            assert layers <= prev_layers or (prev == INF).sum() > (d == INF).sum()
        prev, prev_layers = d, layers


def test_fixed_depth_network():
    m = synth.bernoulli(80, 80, 0.3, 2)
    free = np.flatnonzero(m.reshape(-1) == 0)
    full, layers = oracle.bfs(m, free[:2])
    for L in (1, 5, layers // 2, layers, layers + 4):
        d, got = oracle.bfs(m, free[:2], max_layers=L)
        want = np.where(full <= L, full, INF)
        assert np.array_equal(d, want)
        assert got == min(L, layers)


def _check_path(m, d, s, path):
    H, W = m.shape
    assert path[0] == s
    assert d.reshape(-1)[path[-1]] == 0
    assert len(path) == int(d.reshape(-1)[s]) + 1
    for a, b in zip(path[:-1], path[1:]):
        ay, ax = divmod(int(a), W)
        by, bx = divmod(int(b), W)
        assert max(abs(ay - by), abs(ax - bx)) == 1
        assert not m[by, bx]
        assert d[by, bx] == d[ay, ax] - 1
        # tie-break: no neighbour with a lower linear index also had d - 1
        for dy, dx in NB8:
            ny, nx = ay + dy, ax + dx
            if 0 <= ny < H and 0 <= nx < W and ny * W + nx < b:
                assert m[ny, nx] or d[ny, nx] != d[ay, ax] - 1


@pytest.mark.parametrize("seed", range(20))
def test_trace_invariants_and_tiebreak(seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(2, 60)), int(rng.integers(2, 60))
    m = synth.bernoulli(H, W, 0.3, 50 + seed)
    free = np.flatnonzero(m.reshape(-1) == 0)
    if free.size < 2:
        return
    tg = rng.choice(free, size=min(3, free.size), replace=False)
    st = rng.choice(H * W, size=40)
    d, _ = oracle.bfs(m, tg)
    off, cells, status = oracle.trace(m, d, st)
    ref = dijkstra(m, tg)
    for i, s in enumerate(st):
        p = cells[off[i]:off[i + 1]]
        if m.reshape(-1)[s]:
            assert status[i] == 2 and p.size == 0
        elif d.reshape(-1)[s] == INF:
            assert status[i] == 1 and p.size == 0
        else:
            assert status[i] == 0
            _check_path(m, d, s, p)
            assert p.size - 1 == ref.reshape(-1)[s]          # BFS-optimal step count
            assert p[-1] in set(int(t) for t in tg)


def test_trace_golden_ties():
    cases, cur = [], None
    for line in open(os.path.join(GOLD, "trace_ties.txt")):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "case":
            cur = {"name": f[1]}
            cases.append(cur)
        elif f[0] == "H":
            cur["H"], cur["W"] = int(f[1]), int(f[3])
        else:
            cur[f[0]] = [int(v) for v in f[1:]]
    assert len(cases) == 3
    for c in cases:
        m = np.zeros((c["H"], c["W"]), np.uint8)
        for o in c["obstacles"]:
            m.reshape(-1)[o] = 1
        d, _ = oracle.bfs(m, c["target"])
        off, cells, status = oracle.trace(m, d, c["start"])
        assert status[0] == 0
        assert cells.tolist() == c["path"], c["name"]


def test_errors():
    m = np.zeros((4, 4), np.uint8)
    m[1, 1] = 1
    with pytest.raises(oracle.OracleError) as e:
        oracle.bfs(m, [5])
    assert e.value.code == oracle.EOBSTACLE
    with pytest.raises(oracle.OracleError) as e:
        oracle.bfs(m, [16])
    assert e.value.code == oracle.EINVAL
    with pytest.raises(oracle.OracleError) as e:
        oracle.bfs(m, [])
    assert e.value.code == oracle.EINVAL
    d, layers = oracle.bfs(m, [0, 0, 0])          # duplicates are fine
    assert d[0, 0] == 0 and layers == 4          # (3,3) goes around (1,1)


def test_unreachable_pocket():
    m = np.zeros((7, 7), np.uint8)
    m[2:5, 2] = m[2:5, 4] = m[2, 2:5] = m[4, 2:5] = 1
    d, layers = oracle.bfs(m, [0])
    assert d[3, 3] == INF
    off, cells, status = oracle.trace(m, d, [3 * 7 + 3, 2 * 7 + 2, 48])
    assert status.tolist() == [1, 2, 0]


def test_euclid_diagonal_and_validity():
    z = np.zeros((12, 12), np.uint8)
    d, _ = oracle.bfs(z, [0])
    off, cells, status = oracle.euclid_trace(z, d, [5 * 12 + 5, 11 * 12 + 11])
    assert status.tolist() == [0, 0]
    assert cells[off[0]:off[1]].tolist() == [k * 12 + k for k in range(5, -1, -1)]
    assert cells[off[1]:off[2]].tolist() == [k * 12 + k for k in range(11, -1, -1)]
    # straight axis run stays straight
    off, cells, _ = oracle.euclid_trace(z, d, [7 * 12])
    assert cells.tolist() == [k * 12 for k in range(7, -1, -1)]
    m = synth.bernoulli(60, 60, 0.3, 9)
    free = np.flatnonzero(m.reshape(-1) == 0)
    d, _ = oracle.bfs(m, free[:2])
    st = free[::37]
    off, cells, status = oracle.euclid_trace(m, d, st)
    for i, s in enumerate(st):
        p = cells[off[i]:off[i + 1]]
        if status[i] != 0:
            continue
        assert p[0] == s and d.reshape(-1)[p[-1]] == 0
        assert len(p) <= 2 * int(d.reshape(-1)[s]) + 1
        for a, b in zip(p[:-1], p[1:]):
            ay, ax = divmod(int(a), 60)
            by, bx = divmod(int(b), 60)
            assert max(abs(ay - by), abs(ax - bx)) == 1 and not m[by, bx]


@pytest.mark.parametrize("seed", range(6))
def test_parallel_cpu_baseline_equals_oracle(seed):
    """The OpenMP level-synchronous BFS (the parallel CPU baseline, not the
    oracle) gives the oracle's distances and layer count."""
    rng = np.random.default_rng(100 + seed)
    H, W = (int(v) for v in rng.integers(1, 400, 2))
    kind = seed % 3
    if kind == 0:
        m = synth.bernoulli(H, W, 0.3, 200 + seed)
    elif kind == 1:
        m = synth.dfs_maze(max(H, 3), max(W, 3), 300 + seed)
        H, W = m.shape
    else:
        m = synth.empty(H, W)
    free = np.flatnonzero(m.reshape(-1) == 0)
    t = rng.choice(free, min(free.size, 1 + seed), replace=False).astype(np.uint32)
    d1, l1 = oracle.bfs(m, t)
    d2, l2, threads = oracle.bfs_parallel(m, t)
    assert threads >= 1
    assert l1 == l2 and np.array_equal(d1, d2)


def test_parallel_cpu_baseline_errors():
    m = synth.empty(5, 5)
    m[2, 2] = 1
    with pytest.raises(oracle.OracleError) as e:
        oracle.bfs_parallel(m, np.array([12], np.uint32))
    assert e.value.code == oracle.EOBSTACLE
    with pytest.raises(oracle.OracleError) as e:
        oracle.bfs_parallel(m, np.array([25], np.uint32))
    assert e.value.code == oracle.EINVAL


def read_euclid_golden():
    """Hand-worked Euclidean reconstruction cases (tests/golden/euclid_cases.txt)."""
    cases, cur = [], None
    for line in open(os.path.join(GOLD, "euclid_cases.txt")):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "case":
            cur = {"name": f[1]}
            cases.append(cur)
        elif f[0] == "H":
            cur["H"], cur["W"] = int(f[1]), int(f[3])
        else:
            cur[f[0]] = [int(v) for v in f[1:]]
    for c in cases:
        m = np.zeros((c["H"], c["W"]), np.uint8)
        for o in c["obstacles"]:
            m.reshape(-1)[o] = 1
        c["mask"] = m
    return cases


def test_euclid_golden_plateau_rules():
    """Eq. 1's order, the corner-of-diagonal step, the squeeze step and the
    forward straightening, each pinned by a case worked out by hand."""
    cases = read_euclid_golden()
    assert [c["name"] for c in cases] == ["left_before_up", "corner_step", "corner_blocked_left",
                                          "squeeze"]
    for c in cases:
        d, _ = oracle.bfs(c["mask"], c["targets"])
        off, cells, status = oracle.euclid_trace(c["mask"], d, c["start"])
        assert status.tolist() == [0], c["name"]
        assert cells.tolist() == c["path"], c["name"]
        # the straightened path keeps the raw walk's end-points and order
        raw = c["raw"]
        assert raw[0] == c["path"][0] and raw[-1] == c["path"][-1]
        it = iter(raw)
        assert all(p in it for p in c["path"]), c["name"]
