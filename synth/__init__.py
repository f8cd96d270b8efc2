"""Seeded synthetic workloads for the max-pooling path planner.

Inputs only: obstacle masks (uint8, nonzero = obstacle, row-major H x W),
target cells and start cells (uint32 linear indices y * W + x). Nothing here
computes a distance or a path, so both the CUDA library and the CPU oracle may
consume these arrays.

The five named workloads follow the shapes of the paper's experiments: a small
random grid, generated mazes like the paper's 101 x 101 maze (Results, "oMAP
versus Dijkstra"), many-source maps like its taxi and 26000^2 examples (Results,
"Multi-source Multi-target Path Planning" and "Limitations and Practical
Considerations"). The paper's own maps are not available, so seeded synthetic
grids stand in for them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_SRC = os.path.join(_HERE, "gen.c")
_lock = threading.Lock()
_lib_handle = None


def build(force: bool = False) -> str:
    """Compile gen.c into libsynth.so beside it (gcc, portable C)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    with _lock:
        if _lib_handle is None:
            build()
            L = ctypes.CDLL(_SO)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i64, u64, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            L.synth_subseed.argtypes = [u64, u64]
            L.synth_subseed.restype = u64
            L.synth_rng_stream.argtypes = [u64, u64p, i64]
            L.synth_xoshiro_from_state.argtypes = [u64p, u64p, i64]
            L.synth_splitmix_stream.argtypes = [u64, u64p, i64]
            L.synth_uniform_ints.argtypes = [u64, i64, i64, i64p, i64]
            L.synth_uniform_doubles.argtypes = [u64, ctypes.POINTER(ctypes.c_double), i64]
            L.synth_bernoulli.argtypes = [u8p, i64, i64, dbl, u64]
            L.synth_fill.argtypes = [u8p, i64, ctypes.c_uint8]
            L.synth_dfs_maze.argtypes = [u8p, i64, i64, u64]
            L.synth_dfs_maze.restype = ctypes.c_int
            L.synth_remove_walls.argtypes = [u8p, i64, i64, dbl, u64]
            L.synth_remove_walls.restype = i64
            L.synth_rectangles.argtypes = [u8p, i64, i64, i64, i64, dbl, u64]
            L.synth_rectangles.restype = i64
            L.synth_sample_free.argtypes = [u8p, i64, i64, i64, u64, u32p]
            L.synth_sample_free.restype = i64
            _lib_handle = L
    return _lib_handle


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


# ---- random streams ------------------------------------------------------

def subseed(seed: int, stream: int) -> int:
    return int(_lib().synth_subseed(seed & (2**64 - 1), stream))


def rng_stream(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, np.uint64)
    _lib().synth_rng_stream(seed, _p(out, ctypes.c_uint64), n)
    return out


def xoshiro_from_state(state, n: int) -> np.ndarray:
    st = np.asarray(state, np.uint64)
    out = np.empty(n, np.uint64)
    _lib().synth_xoshiro_from_state(_p(st, ctypes.c_uint64), _p(out, ctypes.c_uint64), n)
    return out


def splitmix_stream(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, np.uint64)
    _lib().synth_splitmix_stream(seed, _p(out, ctypes.c_uint64), n)
    return out


def uniform_ints(seed: int, lo: int, hi: int, n: int) -> np.ndarray:
    out = np.empty(n, np.int64)
    _lib().synth_uniform_ints(seed, lo, hi, _p(out, ctypes.c_int64), n)
    return out


def uniform_doubles(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _lib().synth_uniform_doubles(seed, _p(out, ctypes.c_double), n)
    return out


# ---- grids ---------------------------------------------------------------

def bernoulli(H: int, W: int, p: float, seed: int) -> np.ndarray:
    m = np.empty((H, W), np.uint8)
    _lib().synth_bernoulli(_p(m, ctypes.c_uint8), H, W, p, seed)
    return m


def empty(H: int, W: int) -> np.ndarray:
    return np.zeros((H, W), np.uint8)


def dfs_maze(H: int, W: int, seed: int) -> np.ndarray:
    m = np.empty((H, W), np.uint8)
    if _lib().synth_dfs_maze(_p(m, ctypes.c_uint8), H, W, seed) != 0:
        raise MemoryError("dfs_maze")
    return m


def remove_walls(mask: np.ndarray, frac: float, seed: int) -> int:
    assert mask.flags.c_contiguous and mask.dtype == np.uint8
    H, W = mask.shape
    n = _lib().synth_remove_walls(_p(mask, ctypes.c_uint8), H, W, frac, seed)
    if n < 0:
        raise MemoryError("remove_walls")
    return int(n)


def rectangles(mask: np.ndarray, smin: int, smax: int, cover: float, seed: int) -> int:
    assert mask.flags.c_contiguous and mask.dtype == np.uint8
    H, W = mask.shape
    n = _lib().synth_rectangles(_p(mask, ctypes.c_uint8), H, W, smin, smax, cover, seed)
    if n < 0:
        raise MemoryError("rectangles")
    return int(n)


def sample_free(mask: np.ndarray, k: int, seed: int) -> np.ndarray:
    assert mask.flags.c_contiguous and mask.dtype == np.uint8
    H, W = mask.shape
    out = np.empty(k, np.uint32)
    r = _lib().synth_sample_free(_p(mask, ctypes.c_uint8), H, W, k, seed, _p(out, ctypes.c_uint32))
    if r != k:
        raise ValueError(f"cannot draw {k} distinct free cells")
    return out


# ---- named workloads -----------------------------------------------------

# sub-seed streams of one workload seed
S_GRID, S_WALLS, S_RECTS, S_TARGETS, S_STARTS, S_SHAPE, S_NT, S_NS = 1, 2, 3, 4, 5, 6, 7, 8


@dataclass
class Workload:
    name: str
    mask: np.ndarray              # (H, W) uint8, nonzero = obstacle
    targets: np.ndarray           # uint32 linear indices (paper: sources, I_s = 1)
    starts: np.ndarray            # uint32 linear indices (cells paths are traced from)
    dist_bits: int = 32           # 16 or 32
    meta: dict = field(default_factory=dict)

    @property
    def H(self) -> int:
        return int(self.mask.shape[0])

    @property
    def W(self) -> int:
        return int(self.mask.shape[1])


def c1_small(seed: int = 1) -> Workload:
    """64 x 64, Bernoulli(0.3) obstacles, 1 target, 10 starts, uint16 distances."""
    m = bernoulli(64, 64, 0.3, subseed(seed, S_GRID))
    t = sample_free(m, 1, subseed(seed, S_TARGETS))
    s = sample_free(m, 10, subseed(seed, S_STARTS))
    return Workload("grid64_bernoulli0.3_t1_s10", m, t, s, 16, {"seed": seed})


def c2_maze(seed: int = 2, side: int = 1024) -> Workload:
    """side x side perfect DFS maze (lattice side/2), 4 targets, 100 starts."""
    m = dfs_maze(side, side, subseed(seed, S_GRID))
    t = sample_free(m, 4, subseed(seed, S_TARGETS))
    s = sample_free(m, 100, subseed(seed, S_STARTS))
    return Workload(f"maze{side}_dfs_t4_s100", m, t, s, 32, {"seed": seed})


def c3_maze_open(seed: int = 3, side: int = 4096) -> Workload:
    """side x side DFS maze with 20% of the remaining lattice walls opened,
    1000 targets, 1000 starts."""
    m = dfs_maze(side, side, subseed(seed, S_GRID))
    remove_walls(m, 0.2, subseed(seed, S_WALLS))
    t = sample_free(m, 1000, subseed(seed, S_TARGETS))
    s = sample_free(m, 1000, subseed(seed, S_STARTS))
    return Workload(f"maze{side}_dfs_open20_t1000_s1000", m, t, s, 32, {"seed": seed})


def c4_member(i: int, base_seed: int = 4, side_lo: int = 64, side_hi: int = 2048) -> Workload:
    """Member i of the batched stream: square side uniform in [side_lo, side_hi];
    even i Bernoulli(0.3), odd i DFS maze; 1-16 targets; 10-200 starts."""
    seed = base_seed + i
    S = int(uniform_ints(subseed(seed, S_SHAPE), side_lo, side_hi, 1)[0])
    nt = int(uniform_ints(subseed(seed, S_NT), 1, 16, 1)[0])
    ns = int(uniform_ints(subseed(seed, S_NS), 10, 200, 1)[0])
    if i % 2 == 0:
        m = bernoulli(S, S, 0.3, subseed(seed, S_GRID))
        kind = "bernoulli0.3"
    else:
        m = dfs_maze(S, S, subseed(seed, S_GRID))
        kind = "dfs"
    t = sample_free(m, nt, subseed(seed, S_TARGETS))
    s = sample_free(m, ns, subseed(seed, S_STARTS))
    bits = 16 if S * S <= 65535 else 32
    return Workload(f"batch{i}_{kind}_{S}", m, t, s, bits, {"seed": seed, "index": i})


def c4_batch(n: int = 256, base_seed: int = 4, side_lo: int = 64, side_hi: int = 2048):
    return [c4_member(i, base_seed, side_lo, side_hi) for i in range(n)]


def poisson_arrivals(n: int, rate_per_s: float, seed: int = 4) -> np.ndarray:
    """Arrival times (s) of a Poisson process: exponential gaps by inversion."""
    u = uniform_doubles(subseed(seed, 99), n)
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)


def c5_huge(seed: int = 5, side: int = 23170, n_targets: int = 64, n_starts: int = 4000) -> Workload:
    """side x side Bernoulli(0.25) plus rectangles (sides 16-512) until they
    cover 10% of the area; 64 targets, 4000 starts; uint32 distances."""
    m = bernoulli(side, side, 0.25, subseed(seed, S_GRID))
    rectangles(m, 16, min(512, side), 0.10, subseed(seed, S_RECTS))
    t = sample_free(m, n_targets, subseed(seed, S_TARGETS))
    s = sample_free(m, n_starts, subseed(seed, S_STARTS))
    return Workload(f"grid{side}_bernoulli0.25_rect10_t{n_targets}_s{n_starts}", m, t, s, 32,
                    {"seed": seed})


def open_grid(H: int, W: int, targets, starts, dist_bits: int = 32) -> Workload:
    """Obstacle-free grid with the given end-points (the paper's run-time
    experiments use empty maps)."""
    return Workload(f"empty{H}x{W}", empty(H, W), np.asarray(targets, np.uint32),
                    np.asarray(starts, np.uint32), dist_bits)


CONFIGS = {
    "c1": c1_small,
    "c2": c2_maze,
    "c3": c3_maze_open,
    "c5": c5_huge,
}
