"""CPU oracle for the max-pooling path planner -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never calls it, and it
shares no code with the CUDA library (it has its own C source, its own build
step and its own status constants).

Functions follow the paper's Methods section; see ``oracle.c`` for the
derivation that makes a plain multi-source BFS the exact value of the layer
recurrence. Status codes: 0 ok, 1 invalid argument, 2 out of memory / capacity,
6 target on an obstacle. Distance sentinel: 0xFFFFFFFF.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib_handle = None

INF = 0xFFFFFFFF
OK, EINVAL, ENOMEM, EOBSTACLE = 0, 1, 2, 6


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (gcc, plain C)."""
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
            i8p = ctypes.POINTER(ctypes.c_int8)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64 = ctypes.c_int64
            L.oracle_bfs.argtypes = [u8p, i64, i64, u32p, i64, ctypes.c_uint32, u32p, u32p]
            L.oracle_trace.argtypes = [u8p, u32p, i64, i64, u32p, i64, u64p, u32p, ctypes.c_uint64, i8p]
            L.oracle_omap.argtypes = [u8p, i64, i64, u32p, i64, ctypes.c_int32, i32p]
            L.oracle_euclid_trace.argtypes = [u8p, u32p, i64, i64, u32p, i64, u64p, u32p,
                                              ctypes.c_uint64, i8p]
            for f in (L.oracle_bfs, L.oracle_trace, L.oracle_omap, L.oracle_euclid_trace):
                f.restype = ctypes.c_int
            _lib_handle = L
    return _lib_handle


_PAR_SO = os.path.join(_HERE, "libparbfs.so")
_PAR_SRC = os.path.join(_HERE, "parallel_bfs.c")
_par_handle = None


def build_parallel(force: bool = False) -> str:
    """Compile parallel_bfs.c (the OpenMP CPU baseline, not the oracle)."""
    if force or not os.path.exists(_PAR_SO) or os.path.getmtime(_PAR_SO) < os.path.getmtime(_PAR_SRC):
        tmp = _PAR_SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _PAR_SRC,
                               "-o", tmp])
        os.replace(tmp, _PAR_SO)
    return _PAR_SO


def _par_lib():
    global _par_handle
    with _lock:
        if _par_handle is None:
            build_parallel()
            L = ctypes.CDLL(_PAR_SO)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            L.parallel_bfs.argtypes = [ctypes.POINTER(ctypes.c_uint8), ctypes.c_int64, ctypes.c_int64,
                                       u32p, ctypes.c_int64, u32p, u32p,
                                       ctypes.POINTER(ctypes.c_int32)]
            L.parallel_bfs.restype = ctypes.c_int
            _par_handle = L
    return _par_handle


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _mask(mask) -> np.ndarray:
    m = np.ascontiguousarray(mask)
    if m.dtype != np.uint8:
        m = (m != 0).astype(np.uint8)
    return m


def bfs(mask, targets, max_layers: int = 0):
    """Multi-source 8-neighbour BFS distances (uint32 H x W, INF = unreached
    or obstacle) and the number of layers (largest finite distance)."""
    m = _mask(mask)
    H, W = m.shape
    t = np.ascontiguousarray(targets, np.uint32)
    dist = np.empty((H, W), np.uint32)
    layers = ctypes.c_uint32(0)
    st = _lib().oracle_bfs(_p(m, ctypes.c_uint8), H, W, _p(t, ctypes.c_uint32), t.size,
                           max_layers, _p(dist, ctypes.c_uint32), ctypes.byref(layers))
    if st:
        raise OracleError(st, "oracle_bfs")
    return dist, int(layers.value)


def bfs_parallel(mask, targets):
    """The parallel CPU baseline (level-synchronous BFS on all host cores,
    parallel_bfs.c; not the oracle): distances, layers and the threads used."""
    m = _mask(mask)
    H, W = m.shape
    t = np.ascontiguousarray(targets, np.uint32)
    dist = np.empty((H, W), np.uint32)
    layers = ctypes.c_uint32(0)
    threads = ctypes.c_int32(0)
    st = _par_lib().parallel_bfs(_p(m, ctypes.c_uint8), H, W, _p(t, ctypes.c_uint32), t.size,
                                 _p(dist, ctypes.c_uint32), ctypes.byref(layers), ctypes.byref(threads))
    if st:
        raise OracleError(st, "parallel_bfs")
    return dist, int(layers.value), int(threads.value)


def trace(mask, dist, starts):
    """Simple path reconstruction with the lowest-index tie-break.
    Returns (offsets uint64[n+1], cells uint32[total], status int8[n])."""
    m = _mask(mask)
    H, W = m.shape
    d = np.ascontiguousarray(dist, np.uint32)
    s = np.ascontiguousarray(starts, np.uint32)
    n = s.size
    offsets = np.zeros(n + 1, np.uint64)
    status = np.zeros(max(n, 1), np.int8)
    lens = np.where(m.reshape(-1)[s] != 0, 0,
                    np.where(d.reshape(-1)[s] == INF, 0, d.reshape(-1)[s].astype(np.uint64) + 1))
    cap = int(lens.sum())
    cells = np.zeros(max(cap, 1), np.uint32)
    st = _lib().oracle_trace(_p(m, ctypes.c_uint8), _p(d, ctypes.c_uint32), H, W,
                             _p(s, ctypes.c_uint32), n, _p(offsets, ctypes.c_uint64),
                             _p(cells, ctypes.c_uint32), cap, _p(status, ctypes.c_int8))
    if st:
        raise OracleError(st, "oracle_trace")
    return offsets, cells[:cap], status[:n]


def omap(mask, targets, L: int) -> np.ndarray:
    """The literal layer recurrence after L layers (int32 activity map O)."""
    m = _mask(mask)
    H, W = m.shape
    t = np.ascontiguousarray(targets, np.uint32)
    A = np.empty((H, W), np.int32)
    st = _lib().oracle_omap(_p(m, ctypes.c_uint8), H, W, _p(t, ctypes.c_uint32), t.size, L,
                            _p(A, ctypes.c_int32))
    if st:
        raise OracleError(st, "oracle_omap")
    return A


def euclid_trace(mask, dist, starts):
    """Euclidean path reconstruction (4-neighbour ascent + straightening).
    Returns (offsets, cells, status) with the per-start status of trace()
    (0 path, 1 unreachable, 2 on an obstacle). A walk that finds no next cell
    can only come from a plane that is not a BFS distance map; the call then
    raises OracleError(EINVAL)."""
    m = _mask(mask)
    H, W = m.shape
    d = np.ascontiguousarray(dist, np.uint32)
    s = np.ascontiguousarray(starts, np.uint32)
    n = s.size
    fin = d.reshape(-1)[s]
    cap = int(np.where(fin == INF, 0, 2 * fin.astype(np.uint64) + 1).sum()) + 1
    offsets = np.zeros(n + 1, np.uint64)
    status = np.zeros(max(n, 1), np.int8)
    cells = np.zeros(cap, np.uint32)
    st = _lib().oracle_euclid_trace(_p(m, ctypes.c_uint8), _p(d, ctypes.c_uint32), H, W,
                                    _p(s, ctypes.c_uint32), n, _p(offsets, ctypes.c_uint64),
                                    _p(cells, ctypes.c_uint32), cap, _p(status, ctypes.c_int8))
    if st:
        raise OracleError(st, "oracle_euclid_trace")
    return offsets, cells[: int(offsets[-1])], status[:n]


def distance_from_activity(A: np.ndarray, L: int) -> np.ndarray:
    """First-activation layer from a final activity map after L layers:
    d = L + 1 - O where O > 0, INF elsewhere (the relation the oracle header
    derives from the layer recurrence)."""
    A = np.asarray(A, np.int64)
    return np.where(A > 0, L + 1 - A, INF).astype(np.uint32)
