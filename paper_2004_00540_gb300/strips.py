"""One grid split into row strips over several ranks (one GPU each).

Rank r owns rows [a_r, b_r) of the H x W grid and keeps a plane of distances
over its extended strip: its own rows plus up to k rows of each neighbour
(the halo). A round runs k layers of the wave on the extended strip, resumed
from the plane (mpn_propagate_resume: the paper's recursive mode, which feeds
the activity map of one run into the next; Appendix, Table I). Activity moves
one cell per layer (Methods, "Activity Map Generation"), so after the round
every owned cell with distance up to (j + 1) k is exact, while the halo rows
may be stale; the ranks then swap their edge rows: the top k owned rows go up,
the bottom k down, and replace the neighbours' halos. A round in which no
rank's owned rows gained a cell ends the solve (an OR all-reduce): layers form
a contiguous range, so nothing can be reached later. The result equals the
whole grid solved at once, bit for bit.

The per-strip work runs through an engine with one call, resume(plane, from,
to) -> plane; GpuStripEngine is the library's. Communication goes through a
comm with exchange() and any(): TorchComm (torch.distributed send/recv and
all_reduce; NCCL between GPUs, gloo on CPU), or LocalComms, which runs all
ranks of one process round by round (a host-side emulation for one GPU: the
ranks' kernels never wait on one another).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

INF32 = 0xFFFFFFFF


def strip_rows(H: int, world: int, rank: int, k: int):
    """(a, b, ea, eb): owned rows [a, b) and extended rows [ea, eb) of rank
    `rank`. Every strip owns at least k rows, so a halo never reaches past the
    neighbouring strip."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    if k < 1 or H < world * k:
        raise ValueError(f"{H} rows cannot give {world} strips of at least {k} rows")
    base, extra = divmod(H, world)
    a = rank * base + min(rank, extra)
    b = a + base + (1 if rank < extra else 0)
    return a, b, max(0, a - k), min(H, b + k)


@dataclass
class Strip:
    """One rank's share of the grid and its plane of distances (uint32,
    INF32 = unreached) over the extended strip."""
    mask: np.ndarray          # extended strip's rows of the obstacle mask
    plane: object             # (eb - ea) x W distances: numpy array or torch tensor
    a: int
    b: int
    ea: int
    eb: int
    k: int
    layer: int = 0            # distances up to `layer` are final in the owned rows

    @classmethod
    def make(cls, mask: np.ndarray, targets, world: int, rank: int, k: int, like=None):
        H, W = mask.shape
        a, b, ea, eb = strip_rows(H, world, rank, k)
        plane = np.full((eb - ea, W), INF32, np.uint32)
        t = np.asarray(targets, np.int64)
        y, x = t // W, t % W
        sel = (y >= ea) & (y < eb)
        plane[y[sel] - ea, x[sel]] = 0
        if like is not None:   # a torch device for the plane
            import torch
            plane = torch.from_numpy(plane.view(np.int32)).to(like)
        return cls(np.ascontiguousarray(mask[ea:eb]), plane, a, b, ea, eb, k)

    def own(self):
        return self.plane[self.a - self.ea:self.b - self.ea]

    def step(self, engine, max_layers: int = 0) -> bool:
        """k more layers (capped at max_layers if set); True if an owned cell
        was reached."""
        to = self.layer + self.k
        if max_layers:
            to = min(to, max_layers)
        before = self.own()
        before = before.clone() if hasattr(before, "clone") else before.copy()
        self.plane = engine.resume(self.plane, self.layer, to)
        self.layer = to
        after = self.own()
        if hasattr(after, "clone"):
            return bool((after != before).any().item())
        return bool((after != before).any())

    def halo_out(self):
        """(rows for the rank above, rows for the rank below): the top and
        bottom k owned rows (None at the grid's edge)."""
        up = self.plane[self.a - self.ea:self.a - self.ea + self.k] if self.ea < self.a else None
        dn = self.plane[self.b - self.ea - self.k:self.b - self.ea] if self.eb > self.b else None
        return up, dn

    def halo_in(self, from_up, from_dn):
        """The neighbours' edge rows replace this strip's halo rows."""
        if from_up is not None:
            self.plane[0:self.a - self.ea] = from_up[self.k - (self.a - self.ea):]
        if from_dn is not None:
            self.plane[self.b - self.ea:] = from_dn[:self.eb - self.b]


class TorchComm:
    """Halo exchange and the OR of the ranks' flags over torch.distributed."""

    def __init__(self, dist, rank: int, world: int, device=None):
        self.dist, self.rank, self.world, self.device = dist, rank, world, device

    def exchange(self, strip: Strip):
        import torch
        up, dn = strip.halo_out()
        ops, got_up, got_dn = [], None, None
        if self.rank > 0:
            got_up = torch.empty_like(_as_tensor(up, self.device))
            ops.append(self.dist.P2POp(self.dist.isend, _as_tensor(up, self.device).contiguous(), self.rank - 1))
            ops.append(self.dist.P2POp(self.dist.irecv, got_up, self.rank - 1))
        if self.rank < self.world - 1:
            got_dn = torch.empty_like(_as_tensor(dn, self.device))
            ops.append(self.dist.P2POp(self.dist.isend, _as_tensor(dn, self.device).contiguous(), self.rank + 1))
            ops.append(self.dist.P2POp(self.dist.irecv, got_dn, self.rank + 1))
        if ops:
            for r in self.dist.batch_isend_irecv(ops):
                r.wait()
        strip.halo_in(_like(got_up, strip.plane), _like(got_dn, strip.plane))

    def any(self, flag: bool) -> bool:
        import torch
        t = torch.tensor([1 if flag else 0], dtype=torch.int32, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return bool(t.item())

    def max(self, v: int) -> int:
        import torch
        t = torch.tensor([int(v)], dtype=torch.int64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return int(t.item())


def _as_tensor(a, device):
    import torch
    if hasattr(a, "data_ptr"):
        return a
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(device or "cpu")


def _like(t, plane):
    """A received tensor in the plane's kind (numpy uint32 or torch)."""
    if t is None:
        return None
    if hasattr(plane, "data_ptr"):
        return t.to(plane.device)
    return t.cpu().numpy().view(np.uint32)


def solve_rank(mask: np.ndarray, targets, world: int, rank: int, k: int, engine, comm,
               max_layers: int = 0):
    """Rank `rank`'s part of the split solve: (a, b, owned distances, layer
    count of the whole grid)."""
    s = Strip.make(mask, targets, world, rank, k, like=getattr(engine, "device", None))
    while True:
        changed = s.step(engine, max_layers)
        comm.exchange(s)
        if not comm.any(changed) or (max_layers and s.layer >= max_layers):
            break
    own = s.own()
    own = own.cpu().numpy().view(np.uint32) if hasattr(own, "cpu") else own
    fin = own[own != INF32]
    L = comm.max(int(fin.max()) if fin.size else 0)
    return s.a, s.b, own, L


class LocalComms:
    """All ranks in one process, run round by round: every rank steps, then
    the halos are swapped and the flags ORed (an emulation of the split on one
    device; the ranks' kernels never wait on one another)."""

    @staticmethod
    def solve(mask: np.ndarray, targets, world: int, k: int, engines, max_layers: int = 0):
        strips = [Strip.make(mask, targets, world, r, k, like=getattr(engines[r], "device", None))
                  for r in range(world)]
        while True:
            changed = [s.step(e, max_layers) for s, e in zip(strips, engines)]
            outs = [s.halo_out() for s in strips]
            for r, s in enumerate(strips):
                s.halo_in(outs[r - 1][1] if r > 0 else None, outs[r + 1][0] if r < world - 1 else None)
            if not any(changed) or (max_layers and strips[0].layer >= max_layers):
                break
        H, W = mask.shape
        out = np.empty((H, W), np.uint32)
        for s in strips:
            own = s.own()
            out[s.a:s.b] = own.cpu().numpy().view(np.uint32) if hasattr(own, "cpu") else own
        fin = out[out != INF32]
        return out, int(fin.max()) if fin.size else 0


def gpu_engine(mask: np.ndarray, world: int, rank: int, k: int, device="cuda"):
    """The library engine for rank `rank`'s extended strip."""
    _, _, ea, eb = strip_rows(mask.shape[0], world, rank, k)
    return GpuStripEngine(mask[ea:eb], device)


class GpuStripEngine:
    """The library on one strip: a context over the extended strip's mask,
    resumed from the plane each round (uint32 distances on the device)."""

    def __init__(self, ext_mask: np.ndarray, device="cuda"):
        import torch
        from .mpn import MPN_DIST_U32, mpn_create
        self.device = torch.device(device)
        self._m = torch.from_numpy(np.ascontiguousarray(ext_mask)).to(self.device)
        H, W = ext_mask.shape
        self.ctx = mpn_create(self._m, H, W, MPN_DIST_U32)

    def resume(self, plane, frm: int, to: int):
        import torch
        from .mpn import mpn_get_distances, mpn_propagate_resume
        mpn_propagate_resume(self.ctx, plane, frm, to)
        out = torch.empty_like(plane)
        mpn_get_distances(self.ctx, out)
        return out

    def close(self):
        from .mpn import mpn_destroy
        if self.ctx:
            mpn_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
