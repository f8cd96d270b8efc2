"""Python binding of the C ABI in include/mpn.h (argument marshalling only).

Every function has the C name and forwards to libmpn.so; all work runs in the
library's CUDA kernels. Arrays may be numpy arrays (host memory) or torch
tensors (host or CUDA); CUDA tensors are passed in place. There is no CPU
fallback: if libmpn.so cannot be loaded the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpn.so")

(MPN_OK, MPN_EINVAL, MPN_ENOMEM, MPN_ECUDA, MPN_ETIMEOUT, MPN_EOVERFLOW, MPN_EOBSTACLE, MPN_ESTATE,
 MPN_ECHECK) = range(9)
MPN_DIST_AUTO, MPN_DIST_U16, MPN_DIST_U32 = 0, 16, 32
MPN_UNREACHED16, MPN_UNREACHED32 = 0xFFFF, 0xFFFFFFFF
MPN_PATH_OK, MPN_PATH_UNREACHABLE, MPN_PATH_ON_OBSTACLE = 0, 1, 2

# every symbol include/mpn.h declares
EXPORTS = (
    "mpn_create", "mpn_create_packed", "mpn_set_mask", "mpn_set_stream", "mpn_propagate",
    "mpn_propagate_plain", "mpn_get_distances", "mpn_get_distances_async", "mpn_get_activity",
    "mpn_trace_lengths", "mpn_trace", "mpn_sync", "mpn_destroy", "mpn_status_str", "mpn_set_tuning",
    "mpn_variant_info", "mpn_get_stats", "mpn_launch_count", "mpn_propagate_noalloc",
    "mpn_batch_create", "mpn_batch_set_depth", "mpn_batch_set_mode", "mpn_batch_submit", "mpn_batch_run",
    "mpn_batch_poll", "mpn_batch_wait", "mpn_batch_result", "mpn_batch_info", "mpn_batch_release",
    "mpn_batch_stats", "mpn_batch_destroy", "mpn_autotune", "mpn_trace_euclid",
    "mpn_nearest_targets", "mpn_last_error", "mpn_tune_query", "mpn_propagate_resume", "mpn_check",
)
MPN_BATCH_PENDING, MPN_BATCH_DONE, MPN_BATCH_FAILED = 0, 1, 2


class MPNError(RuntimeError):
    def __init__(self, status: int, what: str):
        detail = ""
        if status in (2, 3) and _lib is not None:
            detail = _lib.mpn_last_error().decode()
        super().__init__(f"{what}: {status_name(status)} ({status})" + (f" [{detail}]" if detail else ""))
        self.status = status


class mpn_stats(ctypes.Structure):
    _fields_ = [
        ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("pitch_words", ctypes.c_int32),
        ("dist_bits", ctypes.c_int32), ("variant", ctypes.c_int32), ("depth", ctypes.c_int32),
        ("tiles_x", ctypes.c_int32), ("tiles_y", ctypes.c_int32), ("blocks", ctypes.c_int32),
        ("layers", ctypes.c_uint32), ("sweeps", ctypes.c_uint32), ("tile_visits", ctypes.c_uint64),
        ("ms_encode", ctypes.c_float), ("ms_propagate", ctypes.c_float), ("ms_trace", ctypes.c_float),
        ("tile_layers", ctypes.c_uint64), ("log_entries", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class mpn_batch_stats_t(ctypes.Structure):
    _fields_ = [
        ("arena_bytes", ctypes.c_uint64), ("arena_used", ctypes.c_uint64),
        ("tiles_used", ctypes.c_uint64), ("next_sweep", ctypes.c_uint32),
        ("rounds", ctypes.c_uint64), ("sweeps", ctypes.c_uint64),
        ("last_round_ms", ctypes.c_float), ("blocks", ctypes.c_int32),
        ("admitted", ctypes.c_int32), ("running", ctypes.c_int32), ("done", ctypes.c_int32),
        ("failed", ctypes.c_int32), ("graph", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH, build_if_missing: bool = True):
    """Load libmpn.so (building it with nvcc first if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path) and build_if_missing:
            from . import build as _b
            _b.build()
        if not os.path.exists(path):
            raise ImportError(f"libmpn.so not found at {path}; run paper_2004_00540_gb300/build.py")
        L = ctypes.CDLL(path)
        vp, i32, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
        pp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "mpn_create": ([vp, i32, i32, i32, vp, pp], ctypes.c_int),
            "mpn_create_packed": ([vp, i32, i32, i32, i32, vp, pp], ctypes.c_int),
            "mpn_set_mask": ([vp, vp], ctypes.c_int),
            "mpn_set_stream": ([vp, vp], ctypes.c_int),
            "mpn_propagate": ([vp, vp, i32, u32, ctypes.POINTER(u32)], ctypes.c_int),
            "mpn_propagate_plain": ([vp, vp, i32, u32, i32, ctypes.POINTER(u32)], ctypes.c_int),
            "mpn_propagate_resume": ([vp, vp, u32, u32, ctypes.POINTER(u32)], ctypes.c_int),
            "mpn_check": ([vp, ctypes.POINTER(u64)], ctypes.c_int),
            "mpn_get_distances": ([vp, vp, i32], ctypes.c_int),
            "mpn_get_distances_async": ([vp, vp, vp], ctypes.c_int),
            "mpn_get_activity": ([vp, u32, vp, i32], ctypes.c_int),
            "mpn_trace_lengths": ([vp, vp, i32, vp], ctypes.c_int),
            "mpn_trace": ([vp, vp, i32, vp, vp, u64, vp], ctypes.c_int),
            "mpn_sync": ([vp], ctypes.c_int),
            "mpn_destroy": ([vp], None),
            "mpn_status_str": ([ctypes.c_int], ctypes.c_char_p),
            "mpn_set_tuning": ([vp, i32, i32], ctypes.c_int),
            "mpn_variant_info": ([i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)],
                                 ctypes.c_int),
            "mpn_get_stats": ([vp, ctypes.POINTER(mpn_stats)], ctypes.c_int),
            "mpn_launch_count": ([], u64),
            "mpn_tune_query": ([i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)],
                               ctypes.c_int),
            "mpn_propagate_noalloc": ([vp, i32, i32, vp, i32, u32, vp, vp], ctypes.c_int),
            "mpn_batch_create": ([u64, i32, vp, pp], ctypes.c_int),
            "mpn_batch_set_depth": ([vp, i32], ctypes.c_int),
            "mpn_batch_set_mode": ([vp, i32], ctypes.c_int),
            "mpn_batch_submit": ([vp, vp, i32, i32, vp, i32, vp, i32, i32, u32,
                                  ctypes.POINTER(u64)], ctypes.c_int),
            "mpn_batch_run": ([vp, u32, ctypes.POINTER(i32), ctypes.POINTER(i32)], ctypes.c_int),
            "mpn_batch_poll": ([vp, u64, ctypes.POINTER(i32)], ctypes.c_int),
            "mpn_batch_wait": ([vp, u64, u32, ctypes.POINTER(i32)], ctypes.c_int),
            "mpn_batch_result": ([vp, u64, vp, vp, vp, u64, vp, ctypes.POINTER(u32)], ctypes.c_int),
            "mpn_batch_info": ([vp, u64, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                ctypes.POINTER(i32), ctypes.POINTER(u64)], ctypes.c_int),
            "mpn_batch_release": ([vp, u64], ctypes.c_int),
            "mpn_batch_stats": ([vp, ctypes.POINTER(mpn_batch_stats_t)], ctypes.c_int),
            "mpn_batch_destroy": ([vp], None),
            "mpn_trace_euclid": ([vp, vp, i32, vp, vp, u64, vp], ctypes.c_int),
            "mpn_nearest_targets": ([vp, vp, i32, vp, vp], ctypes.c_int),
            "mpn_last_error": ([], ctypes.c_char_p),
            "mpn_autotune": ([vp, vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                              ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def status_name(s: int) -> str:
    names = ["MPN_OK", "MPN_EINVAL", "MPN_ENOMEM", "MPN_ECUDA", "MPN_ETIMEOUT", "MPN_EOVERFLOW",
             "MPN_EOBSTACLE", "MPN_ESTATE", "MPN_ECHECK"]
    return names[s] if 0 <= s < len(names) else f"status {s}"


def _check(st: int, what: str):
    if st != MPN_OK:
        raise MPNError(st, what)


def _ptr(a):
    """(pointer, is_device) of a numpy array or torch tensor (must be contiguous)."""
    if a is None:
        return None, False
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, False
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a.device.type == "cuda"
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- C-named functions -------------------------------------------------

def mpn_create(mask, H: int, W: int, dist_bits: int = MPN_DIST_AUTO, stream=None):
    L = load()
    out = ctypes.c_void_p()
    p, _ = _ptr(mask)
    _check(L.mpn_create(p, H, W, dist_bits, _stream_handle(stream), ctypes.byref(out)), "mpn_create")
    return out


def mpn_create_packed(bits, H: int, W: int, pitch_words: int, dist_bits: int = MPN_DIST_AUTO,
                      stream=None):
    L = load()
    out = ctypes.c_void_p()
    p, _ = _ptr(bits)
    _check(L.mpn_create_packed(p, H, W, pitch_words, dist_bits, _stream_handle(stream),
                               ctypes.byref(out)), "mpn_create_packed")
    return out


def mpn_set_mask(ctx, mask):
    _check(load().mpn_set_mask(ctx, _ptr(mask)[0]), "mpn_set_mask")


def mpn_set_stream(ctx, stream):
    _check(load().mpn_set_stream(ctx, _stream_handle(stream)), "mpn_set_stream")


def mpn_propagate(ctx, targets, max_layers: int = 0, wait: bool = True):
    """Returns the layer count (largest finite distance) when wait, else None."""
    n = int(targets.numel() if hasattr(targets, "numel") else np.asarray(targets).size)
    p, _ = _ptr(targets)
    if wait:
        lr = ctypes.c_uint32(0)
        _check(load().mpn_propagate(ctx, p, n, max_layers, ctypes.byref(lr)), "mpn_propagate")
        return int(lr.value)
    _check(load().mpn_propagate(ctx, p, n, max_layers, None), "mpn_propagate")
    return None


def mpn_propagate_resume(ctx, dist_in, from_layer: int, max_layers: int = 0, wait: bool = True):
    """Continue from a distance plane (cells <= from_layer kept); returns the
    largest distance the new layers reached (0 if none) when wait."""
    p, _ = _ptr(dist_in)
    if wait:
        lr = ctypes.c_uint32(0)
        _check(load().mpn_propagate_resume(ctx, p, from_layer, max_layers, ctypes.byref(lr)),
               "mpn_propagate_resume")
        return int(lr.value)
    _check(load().mpn_propagate_resume(ctx, p, from_layer, max_layers, None), "mpn_propagate_resume")
    return None


def mpn_check(ctx) -> int:
    """Cells of the last propagation's plane that break the distance-map
    invariants (0 for a correct plane)."""
    v = ctypes.c_uint64(0)
    st = load().mpn_check(ctx, ctypes.byref(v))
    if st not in (MPN_OK, MPN_ECHECK):
        raise MPNError(st, "mpn_check")
    return int(v.value)


def mpn_propagate_plain(ctx, targets, max_layers: int = 0, check_every: int = 1):
    n = int(targets.numel() if hasattr(targets, "numel") else np.asarray(targets).size)
    lr = ctypes.c_uint32(0)
    _check(load().mpn_propagate_plain(ctx, _ptr(targets)[0], n, max_layers, check_every,
                                      ctypes.byref(lr)), "mpn_propagate_plain")
    return int(lr.value)


def mpn_get_distances(ctx, out):
    p, dev = _ptr(out)
    _check(load().mpn_get_distances(ctx, p, int(dev)), "mpn_get_distances")
    return out


def mpn_get_distances_async(ctx, out, stream=None):
    """Enqueue the distance download on `stream` (None: the context's own) and
    return; `out` is valid once that stream has passed the copy (mpn_sync)."""
    _check(load().mpn_get_distances_async(ctx, _ptr(out)[0], _stream_handle(stream)),
           "mpn_get_distances_async")
    return out


def mpn_get_activity(ctx, L: int, out):
    p, dev = _ptr(out)
    _check(load().mpn_get_activity(ctx, L, p, int(dev)), "mpn_get_activity")
    return out


def mpn_trace_lengths(ctx, starts, offsets):
    n = int(starts.numel() if hasattr(starts, "numel") else np.asarray(starts).size)
    _check(load().mpn_trace_lengths(ctx, _ptr(starts)[0], n, _ptr(offsets)[0]), "mpn_trace_lengths")
    return offsets


def mpn_trace(ctx, starts, offsets, cells, cells_cap: int, status):
    """Returns the status code (MPN_OK or MPN_ENOMEM when cells is too small)."""
    n = int(starts.numel() if hasattr(starts, "numel") else np.asarray(starts).size)
    st = load().mpn_trace(ctx, _ptr(starts)[0], n, _ptr(offsets)[0], _ptr(cells)[0], cells_cap,
                          _ptr(status)[0])
    if st not in (MPN_OK, MPN_ENOMEM):
        raise MPNError(st, "mpn_trace")
    return st


def mpn_trace_euclid(ctx, starts, offsets, cells, cells_cap: int, status):
    """Euclidean reconstruction; returns MPN_OK or MPN_ENOMEM (offsets filled)."""
    n = int(starts.numel() if hasattr(starts, "numel") else np.asarray(starts).size)
    st = load().mpn_trace_euclid(ctx, _ptr(starts)[0], n, _ptr(offsets)[0], _ptr(cells)[0],
                                 cells_cap, _ptr(status)[0])
    if st not in (MPN_OK, MPN_ENOMEM):
        raise MPNError(st, "mpn_trace_euclid")
    return st


def mpn_nearest_targets(ctx, starts, target, dist=None):
    n = int(starts.numel() if hasattr(starts, "numel") else np.asarray(starts).size)
    _check(load().mpn_nearest_targets(ctx, _ptr(starts)[0], n, _ptr(target)[0],
                                      _ptr(dist)[0] if dist is not None else None),
           "mpn_nearest_targets")
    return target


def mpn_sync(ctx):
    _check(load().mpn_sync(ctx), "mpn_sync")


def mpn_destroy(ctx):
    if ctx:
        load().mpn_destroy(ctx)


def mpn_status_str(s: int) -> str:
    return load().mpn_status_str(s).decode()


def mpn_set_tuning(ctx, variant: int, depth: int):
    _check(load().mpn_set_tuning(ctx, variant, depth), "mpn_set_tuning")


def mpn_variant_info(v: int):
    r, w, t = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    st = load().mpn_variant_info(v, ctypes.byref(r), ctypes.byref(w), ctypes.byref(t))
    if st != MPN_OK:
        return None
    return {"region_rows": r.value, "region_words": w.value, "threads": t.value}


def mpn_get_stats(ctx) -> dict:
    s = mpn_stats()
    _check(load().mpn_get_stats(ctx, ctypes.byref(s)), "mpn_get_stats")
    return s.as_dict()


def mpn_autotune(ctx, targets):
    """Measure every tile shape x depth; returns (variant, depth, ms)."""
    n = int(targets.numel() if hasattr(targets, "numel") else np.asarray(targets).size)
    v, d, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(load().mpn_autotune(ctx, _ptr(targets)[0], n, ctypes.byref(v), ctypes.byref(d),
                               ctypes.byref(ms)), "mpn_autotune")
    return v.value, d.value, ms.value


def mpn_tune_query(H: int, W: int, variant: int):
    """(depth, ms) the autotuner recorded for this size bucket and tile shape,
    or None if nothing was measured for it."""
    d, ms = ctypes.c_int32(), ctypes.c_float()
    st = load().mpn_tune_query(H, W, variant, ctypes.byref(d), ctypes.byref(ms))
    if st == MPN_ESTATE:
        return None
    _check(st, "mpn_tune_query")
    return d.value, ms.value


def mpn_launch_count() -> int:
    return int(load().mpn_launch_count())


def mpn_propagate_noalloc(mask, H: int, W: int, targets, dist, max_layers: int = 0,
                          stream=None):
    """Distances into the caller's device buffer `dist` (H*W uint32) with no
    allocation; mask (H*W uint8), targets (32-bit indices) and dist must be
    CUDA tensors. Returns the status code (MPN_OK, MPN_EINVAL past 2048 x
    2048, ...). Raises ValueError/TypeError for buffers the kernels cannot
    use in place (host memory, wrong element size, too few elements)."""
    for name, a in (("mask", mask), ("targets", targets), ("dist", dist)):
        if not hasattr(a, "data_ptr") or a.device.type != "cuda":
            raise TypeError(f"mpn_propagate_noalloc: {name} must be a CUDA tensor")
        if not a.is_contiguous():
            raise ValueError(f"mpn_propagate_noalloc: {name} must be contiguous")
    if H < 1 or W < 1:
        raise ValueError("mpn_propagate_noalloc: H and W must be >= 1")
    if mask.element_size() != 1 or mask.numel() < H * W:
        raise ValueError("mpn_propagate_noalloc: mask must hold H*W bytes")
    if dist.element_size() != 4 or dist.numel() < H * W:
        raise ValueError("mpn_propagate_noalloc: dist must hold H*W 32-bit elements")
    if targets.element_size() != 4:
        raise ValueError("mpn_propagate_noalloc: targets must be 32-bit indices")
    n = int(targets.numel())
    return int(load().mpn_propagate_noalloc(mask.data_ptr(), H, W, targets.data_ptr(), n,
                                            max_layers, dist.data_ptr(), _stream_handle(stream)))


# ---- convenience wrapper -----------------------------------------------

@dataclass
class Paths:
    offsets: np.ndarray   # uint64[n+1]
    cells: np.ndarray     # uint32[offsets[-1]]
    status: np.ndarray    # int8[n]

    def path(self, i: int) -> np.ndarray:
        return self.cells[int(self.offsets[i]):int(self.offsets[i + 1])]


class Planner:
    """One grid resident on the GPU: encode once, propagate and trace many times."""

    def __init__(self, mask, dist_bits: int = MPN_DIST_AUTO, stream=None):
        shape = tuple(mask.shape)
        if len(shape) != 2:
            raise ValueError("mask must be 2-D (H, W)")
        self.H, self.W = int(shape[0]), int(shape[1])
        self.ctx = mpn_create(mask, self.H, self.W, dist_bits, stream)
        self.dist_bits = mpn_get_stats(self.ctx)["dist_bits"]
        self.layers = None

    def close(self):
        if self.ctx:
            mpn_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_tuning(self, variant: int, depth: int):
        mpn_set_tuning(self.ctx, variant, depth)

    def autotune(self, targets):
        t = np.ascontiguousarray(targets, np.uint32) if not hasattr(targets, "data_ptr") else targets
        return mpn_autotune(self.ctx, t)

    def propagate(self, targets, max_layers: int = 0, plain: bool = False, check_every: int = 1):
        t = np.ascontiguousarray(targets, np.uint32) if not hasattr(targets, "data_ptr") else targets
        if plain:
            self.layers = mpn_propagate_plain(self.ctx, t, max_layers, check_every)
        else:
            self.layers = mpn_propagate(self.ctx, t, max_layers)
        return self.layers

    def distances(self) -> np.ndarray:
        out = np.empty((self.H, self.W), np.uint16 if self.dist_bits == 16 else np.uint32)
        return mpn_get_distances(self.ctx, out)

    def activity(self, L: int = 0) -> np.ndarray:
        out = np.empty((self.H, self.W), np.int32)
        return mpn_get_activity(self.ctx, L, out)

    def trace(self, starts) -> Paths:
        s = np.ascontiguousarray(starts, np.uint32)
        n = s.size
        offsets = np.zeros(n + 1, np.uint64)
        mpn_trace_lengths(self.ctx, s, offsets)
        total = int(offsets[-1])
        cells = np.zeros(max(total, 1), np.uint32)
        status = np.zeros(max(n, 1), np.int8)
        st = mpn_trace(self.ctx, s, offsets, cells, total, status)
        if st != MPN_OK:
            raise MPNError(st, "mpn_trace")
        return Paths(offsets, cells[:total], status[:n])

    def nearest_targets(self, starts):
        """(target cell, distance) per start; 0xFFFFFFFF where there is no path."""
        s = np.ascontiguousarray(starts, np.uint32)
        t = np.empty(s.size, np.uint32)
        d = np.empty(s.size, np.uint32)
        mpn_nearest_targets(self.ctx, s, t, d)
        return t, d

    def trace_euclid(self, starts) -> Paths:
        s = np.ascontiguousarray(starts, np.uint32)
        n = s.size
        offsets = np.zeros(n + 1, np.uint64)
        status = np.zeros(max(n, 1), np.int8)
        cells = np.zeros(1, np.uint32)
        mpn_trace_euclid(self.ctx, s, offsets, cells, 0, status)     # sizes first
        total = int(offsets[-1])
        cells = np.zeros(max(total, 1), np.uint32)
        st = mpn_trace_euclid(self.ctx, s, offsets, cells, total, status)
        if st != MPN_OK:
            raise MPNError(st, "mpn_trace_euclid")
        return Paths(offsets, cells[:total], status[:n])

    def stats(self) -> dict:
        return mpn_get_stats(self.ctx)


# ---- batched / continuously batched solving ------------------------------

class Batch:
    """Many grids on one GPU: admission by device memory, rounds of one
    persistent launch over every admitted grid (see include/mpn.h)."""

    def __init__(self, budget_bytes: int, variant: int = -1, stream=None):
        self.h = ctypes.c_void_p()
        _check(load().mpn_batch_create(budget_bytes, variant, _stream_handle(stream),
                                       ctypes.byref(self.h)), "mpn_batch_create")

    def close(self):
        if self.h:
            load().mpn_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_depth(self, depth: int):
        _check(load().mpn_batch_set_depth(self.h, depth), "mpn_batch_set_depth")

    def set_mode(self, per_grid_clock: bool):
        """True: every grid keeps its own sweep clock (see include/mpn.h)."""
        _check(load().mpn_batch_set_mode(self.h, 1 if per_grid_clock else 0), "mpn_batch_set_mode")

    def submit(self, mask, targets, starts, dist_bits: int = MPN_DIST_AUTO, max_layers: int = 0):
        """Ticket, or None when the grid does not fit in the arena now."""
        H, W = int(mask.shape[0]), int(mask.shape[1])
        t = targets if hasattr(targets, "data_ptr") else np.ascontiguousarray(targets, np.uint32)
        s = starts if hasattr(starts, "data_ptr") else np.ascontiguousarray(starts, np.uint32)
        nt = int(t.numel() if hasattr(t, "numel") else t.size)
        ns = int(s.numel() if hasattr(s, "numel") else s.size)
        tk = ctypes.c_uint64(0)
        st = load().mpn_batch_submit(self.h, _ptr(mask)[0], H, W, _ptr(t)[0], nt, _ptr(s)[0], ns,
                                     dist_bits, max_layers, ctypes.byref(tk))
        if st == MPN_ENOMEM:
            return None
        _check(st, "mpn_batch_submit")
        return int(tk.value)

    def run(self, max_sweeps: int = 0):
        """One round; returns (grids still in flight, grids finished)."""
        r, d = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(load().mpn_batch_run(self.h, max_sweeps, ctypes.byref(r), ctypes.byref(d)),
               "mpn_batch_run")
        return r.value, d.value

    def poll(self, ticket: int) -> int:
        s = ctypes.c_int32(0)
        st = load().mpn_batch_poll(self.h, ticket, ctypes.byref(s))
        if s.value == MPN_BATCH_FAILED:
            return MPN_BATCH_FAILED
        _check(st, "mpn_batch_poll")
        return s.value

    def wait(self, ticket: int, max_sweeps: int = 0) -> int:
        """Run rounds until grid `ticket` is done or failed; its state."""
        s = ctypes.c_int32(0)
        st = load().mpn_batch_wait(self.h, ticket, max_sweeps, ctypes.byref(s))
        if s.value == MPN_BATCH_FAILED:
            return MPN_BATCH_FAILED
        _check(st, "mpn_batch_wait")
        return s.value

    def error(self, ticket: int) -> int:
        s = ctypes.c_int32(0)
        return int(load().mpn_batch_poll(self.h, ticket, ctypes.byref(s)))

    def info(self, ticket: int) -> dict:
        H, W, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        tot = ctypes.c_uint64()
        _check(load().mpn_batch_info(self.h, ticket, ctypes.byref(H), ctypes.byref(W),
                                     ctypes.byref(b), ctypes.byref(tot)), "mpn_batch_info")
        return {"H": H.value, "W": W.value, "dist_bits": b.value, "total_cells": tot.value}

    def result(self, ticket: int, n_starts: int, want_dist: bool = True, cells=None,
               offsets=None, status=None):
        """(dist or None, Paths, layers) of a finished grid. The path arrays
        go into the given buffers when passed (numpy arrays or torch tensors,
        host -- page-locked is fastest -- or device; cells must hold the
        grid's total path cells, offsets n_starts + 1 uint64, status n_starts
        int8), else into new host arrays."""
        inf = self.info(ticket)
        dist = None
        if want_dist:
            dist = np.empty((inf["H"], inf["W"]), np.uint16 if inf["dist_bits"] == 16 else np.uint32)
        total = inf["total_cells"]
        off = np.empty(n_starts + 1, np.uint64) if offsets is None else offsets
        cl = np.empty(max(total, 1), np.uint32) if cells is None else cells
        sts = np.empty(max(n_starts, 1), np.int8) if status is None else status
        cap = int(cl.numel() if hasattr(cl, "numel") else cl.size)
        layers = ctypes.c_uint32(0)
        _check(load().mpn_batch_result(self.h, ticket, _ptr(dist)[0] if dist is not None else None,
                                       _ptr(off)[0], _ptr(cl)[0], cap, _ptr(sts)[0],
                                       ctypes.byref(layers)), "mpn_batch_result")
        return dist, Paths(off, cl[:total], sts[:n_starts]), int(layers.value)

    def release(self, ticket: int):
        _check(load().mpn_batch_release(self.h, ticket), "mpn_batch_release")

    def stats(self) -> dict:
        s = mpn_batch_stats_t()
        _check(load().mpn_batch_stats(self.h, ctypes.byref(s)), "mpn_batch_stats")
        return s.as_dict()
