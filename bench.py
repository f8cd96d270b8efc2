#!/usr/bin/env python3
"""Benchmark of the max-pooling path planner on one GB300 (or N, one process
per GPU, each solving its own copy of the workload).

A step is one pass of the whole hot path over the 23170 x 23170 grid
(Bernoulli(0.25) obstacles plus rectangles covering 10 %, 64 targets, 4000
starts): encode the uint8 mask to bits, propagate the activity wave to
convergence, trace all 4000 paths. Inputs are resident in HBM when the timed
region starts (value); e2e repeats the step through the C ABI from pinned host
buffers, with the mask upload and the distance-map and path downloads inside
the timed region, as a stream of solves pipelined over two contexts (one
solve's download overlapping the next one's upload and kernels); e2e.serial
runs them one at a time.

metric: effective cell-updates/s = H * W * L / t, L = the number of layers the
paper's network needs (the largest finite distance), as in the paper's O(N L)
complexity (Methods, "Determining the number of layers L").

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs the same step on its own GPU; rank 0 prints one
JSON line with the max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "effective cell-updates/sec"
UNIT = "cell-updates/s"
BYTES_PER_UPDATE_U32 = 8.125      # read the mask bit, read and write the uint32 distance
# Floor of one propagation: read the packed mask once (1/8 B per cell) and
# write the uint32 distance plane once (4 B per cell); every other byte a
# kernel moves is overhead of its design.
FLOOR_BYTES_PER_CELL_U32 = 4.125
L2_NOTE = "inputs larger than L2 (uint8 mask 537 MB + uint32 distance plane 2.15 GB per step)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--side", type=int, default=23170, help="grid side (default: the full workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--variant", type=int, default=-1, help="tile shape (default: autotuned)")
    ap.add_argument("--depth", type=int, default=32)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-maze batched/served part")
    ap.add_argument("--no-per-config", action="store_true",
                    help="skip the 64^2, 1024^2-maze and 4096^2-maze single-grid timings")
    ap.add_argument("--batch-n", type=int, default=256)
    ap.add_argument("--plain-sample", type=int, default=32,
                    help="mazes timed with one launch per layer (the slow baseline)")
    ap.add_argument("--fig5", action="store_true",
                    help="the paper's run-time experiment on empty n x n grids with fixed L")
    ap.add_argument("--table1", action="store_true",
                    help="one launch per layer (the paper's recursive mode) vs the persistent "
                         "kernel on a 2000 x 2000 grid and on the 1024 x 1024 maze")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.idx = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = ("paper_2004_00540_gb300/csrc/wave.cuh", "paper_2004_00540_gb300/csrc/propagate.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_propagate_traffic.json")


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(workload: str, variant: int, depth: int):
    """DRAM bytes per propagation (k_propagate + k_log_decode launch) from the
    committed ncu capture, or
    None when the kernel sources changed since it was taken, or the capture
    was of another workload or tiling."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
    except Exception:
        return None
    if (t.get("source_sha256") != kernel_source_hash() or t.get("workload") != workload
            or t.get("variant") != variant or t.get("depth") != depth):
        return None
    return t.get("dram_bytes_per_launch")


def shard(n_items: int, rank: int, world: int):
    """Indices of the independent problems rank `rank` of `world` solves
    (round robin; the ranks never exchange data)."""
    return list(range(rank, n_items, world))


def aggregate(local_ms: float, units_per_rank: float, steps: int, world: int, dist=None, device=None):
    """Whole-job time = the slowest rank's time (all-reduce MAX); value =
    the units all ranks processed / that time."""
    t = local_ms
    if dist is not None and world > 1:
        import torch
        tt = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return t, world * units_per_rank * steps / (t * 1e-3)


def workload(side: int):
    if side == 23170:
        return synth.c5_huge()
    return synth.c5_huge(side=side)


def crop(w, side):
    """Top-left side x side window of a workload (end-points that fall inside)."""
    m = np.ascontiguousarray(w.mask[:side, :side])
    def keep(idx):
        y, x = idx // w.W, idx % w.W
        ok = (y < side) & (x < side)
        return (y[ok] * side + x[ok]).astype(np.uint32)
    t = keep(w.targets.astype(np.int64))
    s = keep(w.starts.astype(np.int64))
    return synth.Workload(f"{w.name}_crop{side}", m, t, s, 32, dict(w.meta))


def time_oracle(w, reps=1):
    """The CPU oracle as it stands: BFS + trace, single thread."""
    import oracle
    best = None
    L = 0
    for _ in range(reps):
        t0 = time.perf_counter()
        d, L = oracle.bfs(w.mask, w.targets)
        oracle.trace(w.mask, d, w.starts)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return best, L


def cpu_baseline(w, sample_side=23170):
    s = crop(w, sample_side) if sample_side < w.H else w
    dt, L = time_oracle(s)
    out = {"value": s.H * s.W * L / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"top-left {s.H}x{s.W} window of the workload with the {s.targets.size} targets "
                     f"and {s.starts.size} starts inside it (L={L}); single-thread BFS + trace, "
                     f"{dt:.1f} s", "seconds": dt, "host_cores": os.cpu_count()}
    # the parallel CPU baseline (level-synchronous BFS on all host cores),
    # median of three runs, its distances checked against the oracle's
    import oracle
    want, _ = oracle.bfs(s.mask, s.targets)
    runs, same, threads, Lp = [], True, 0, 0
    for _ in range(3):
        t0 = time.perf_counter()
        d, Lp, threads = oracle.bfs_parallel(s.mask, s.targets)
        runs.append(time.perf_counter() - t0)
        same = same and Lp == L and bool(np.array_equal(d, want))
    tp = statistics.median(runs)
    out["parallel"] = {"value": s.H * s.W * Lp / tp, "unit": UNIT, "cores": threads,
                       "kind": "openmp level-synchronous BFS (no trace)", "seconds": tp,
                       "equals_oracle": same}
    return out


def workload_config(w, layers: int, path_cells: int, world: int) -> dict:
    """The `config` of a bench line: the workload alone (both arms print the
    same dict for the same work; tiling choices go elsewhere)."""
    return {"workload": w.name, "H": w.H, "W": w.W, "targets": int(w.targets.size),
            "starts": int(w.starts.size), "layers": int(layers), "path_cells": int(path_cells),
            "step": "encode + propagate + trace", "parallelism": f"replicas x{world}",
            "l2": L2_NOTE}


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle as it stands (single-thread BFS +
    trace) on the same full workload as a step of our arm. Its W warm-up
    steps run on a 4096 x 4096 window (untimed; only the timed steps count),
    so that K = 20 timed steps of about 10 s each end within a few minutes."""
    if rank != 0:
        return 0
    import oracle
    w = workload(args.side)
    warm = crop(w, min(4096, w.H))
    for _ in range(args.warmup):
        time_oracle(warm)
    times, L, cells = [], 0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        d, L = oracle.bfs(w.mask, w.targets)
        off, _, _ = oracle.trace(w.mask, d, w.starts)
        times.append(time.perf_counter() - t0)
        cells = int(off[-1])
    t = sum(times)
    v = w.H * w.W * L * len(times) / t
    sample = (f"the full {w.H}x{w.W} workload, {w.targets.size} targets, {w.starts.size} starts "
              f"(L={L}), every timed step; warm-up steps on its top-left {warm.H}x{warm.W} window")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": workload_config(w, L, cells, 1),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_per_config(pkg, torch, reps: int = 5):
    """The single-grid configurations besides the headline one (64 x 64
    Bernoulli, the 1024 x 1024 DFS maze, the 4096 x 4096 maze with 20 % of its
    walls opened), device-resident: propagate + trace, best of `reps` after a
    warm-up, each checked against the CPU oracle once (layer count and path
    cell total)."""
    import oracle
    out = {}
    for w in (synth.c1_small(), synth.c2_maze(), synth.c3_maze_open()):
        m = torch.from_numpy(w.mask).cuda()
        t = torch.from_numpy(w.targets.view(np.int32)).cuda()
        s = torch.from_numpy(w.starts.view(np.int32)).cuda()
        n = w.starts.size
        with pkg.Planner(m, w.dist_bits) as pl:
            L = pl.propagate(t)
            off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
            pkg.mpn_trace_lengths(pl.ctx, s, off)
            total = int(off[-1].item())
            cells = torch.zeros(max(total, 1), dtype=torch.int32, device="cuda")
            status = torch.zeros(n, dtype=torch.int8, device="cuda")
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            best, prop, trace = None, None, None
            for r in range(reps + 1):
                torch.cuda.synchronize()
                ev0.record()
                pkg.mpn_propagate(pl.ctx, t, 0, wait=False)
                pkg.mpn_trace(pl.ctx, s, off, cells, total, status)
                ev1.record()
                ev1.synchronize()
                ms = ev0.elapsed_time(ev1)
                st = pl.stats()
                if r and (best is None or ms < best):
                    best, prop, trace = ms, st["ms_propagate"], st["ms_trace"]
        od, oL = oracle.bfs(w.mask, w.targets)
        ooff, _, _ = oracle.trace(w.mask, od, w.starts)
        out[w.name] = {"H": w.H, "W": w.W, "layers": int(L), "dist_bits": w.dist_bits,
                       "step_ms": best, "propagate_ms": prop, "trace_ms": trace,
                       "effective_cell_updates_per_s": w.H * w.W * L / (prop * 1e-3),
                       "paths": int(n), "path_cells": total, "sweeps": st["sweeps"],
                       "variant": st["variant"], "depth": st["depth"],
                       "equals_oracle": bool(L == oL and total == int(ooff[-1]))}
    return out


def autotune_buckets(ws, dev, pkg):
    """Before the batched leg (outside its timed region): the autotuner on one
    grid per size bucket ceil(log2(side)) -- the smallest DFS maze of the
    bucket, the kind whose many layers set the batch's time -- so that the
    batch takes each bucket's measured depth for its tile shape (shape 0)."""
    pick = {}
    for i, w in enumerate(ws):
        b = int(np.ceil(np.log2(max(w.H, w.W))))
        if i % 2 == 1 and (b not in pick or w.H * w.W < ws[pick[b]].H * ws[pick[b]].W):
            pick[b] = i
    tuned = {}
    for b in sorted(pick):
        i = pick[b]
        w = ws[i]
        m, t, _ = dev[i]
        with pkg.Planner(m, w.dist_bits) as pl:
            v, d, ms = pl.autotune(t)
        q = pkg.mpn_tune_query(w.H, w.W, 0)
        tuned[str(b)] = {"grid": w.name, "side": w.H, "best_variant": v, "best_depth": d,
                         "best_ms": ms, "batch_shape0_depth": q[0] if q else None,
                         "batch_shape0_ms": q[1] if q else None}
    return tuned


def run_batched(args, pkg, torch):
    """The 256-maze stream: batched capacity, per-maze baselines, serving."""
    from paper_2004_00540_gb300.serve import Request, serve
    ws = synth.c4_batch(args.batch_n)
    cells = sum(w.H * w.W for w in ws)
    dev = [(torch.from_numpy(w.mask).cuda(), torch.from_numpy(w.targets.view(np.int32)).cuda(),
            torch.from_numpy(w.starts.view(np.int32)).cuda()) for w in ws]
    torch.cuda.synchronize()
    budget = int(sum(w.H * w.W * 5 + 4096 * 64 for w in ws) * 1.5) + (256 << 20)
    out = {"workload": f"{len(ws)} grids, side U{{64..2048}}, even Bernoulli(0.3) / odd DFS maze, "
                       f"1-16 targets, 10-200 starts", "cells": int(cells)}
    out["tuned"] = autotune_buckets(ws, dev, pkg)

    # page-locked host buffers for every grid's paths, allocated once and
    # sized by the warm-up run (as a serving process keeps its response
    # buffers); every timed run still downloads all paths into them
    host = {}

    def batched_once():
        with pkg.Batch(budget) as b:
            t0 = time.perf_counter()
            tks = [b.submit(m, t, s, w.dist_bits) for (m, t, s), w in zip(dev, ws)]
            assert all(tk is not None for tk in tks)
            b.run(0)
            if host:
                res = []
                for i, (tk, w) in enumerate(zip(tks, ws)):
                    a, e = host["cell_at"][i], host["cell_at"][i + 1]
                    o = host["off_at"][i]
                    res.append(b.result(tk, w.starts.size, want_dist=False, cells=host["cells"][a:max(e, a + 1)],
                                        offsets=host["off"][o:o + w.starts.size + 1],
                                        status=host["status"][o:o + max(w.starts.size, 1)]))
            else:
                res = [b.result(tk, w.starts.size, want_dist=False) for tk, w in zip(tks, ws)]
            dt = time.perf_counter() - t0
            st = b.stats()
            totals = [b.info(tk)["total_cells"] for tk in tks]
        return dt, res, st, totals

    _, _, _, totals = batched_once()                 # warm-up
    cell_at = np.concatenate([[0], np.cumsum([max(x, 1) for x in totals])]).astype(np.int64)
    off_at = np.concatenate([[0], np.cumsum([w.starts.size + 1 for w in ws])]).astype(np.int64)
    host.update(cells=torch.empty(int(cell_at[-1]), dtype=torch.int32).pin_memory(),
                off=torch.empty(int(off_at[-1]), dtype=torch.int64).pin_memory(),
                status=torch.empty(int(off_at[-1]), dtype=torch.int8).pin_memory(),
                cell_at=cell_at.tolist(), off_at=off_at.tolist())
    runs = [batched_once() for _ in range(3)]        # the host-side download varies run to run
    dt, res, st, _ = min(runs, key=lambda r: r[0])
    out["batched"] = {"mazes_per_s": len(ws) / dt, "seconds": dt, "rounds": st["rounds"],
                      "sweeps": st["sweeps"], "propagate_round_ms": st["last_round_ms"],
                      "path_cells": int(sum(totals)), "scheduling": "per-grid sweep clocks",
                      "seconds_each": [r[0] for r in runs],
                      "note": "best of 3: submit + one round to convergence + every grid's paths, "
                              "offsets and status downloaded into page-locked host buffers"}

    # per grid, one persistent launch each (same library, no batching)
    t0 = time.perf_counter()
    layers = []
    for (m, t, s), w in zip(dev, ws):
        with pkg.Planner(m, w.dist_bits) as pl:
            layers.append(pl.propagate(t))
            p = pl.trace(s.cpu().numpy().view(np.uint32))
    dts = time.perf_counter() - t0
    out["per_maze_persistent"] = {"mazes_per_s": len(ws) / dts, "seconds": dts}
    # exactness: batched paths == per-grid paths
    for (_, paths, L), Lr in zip(res[:8], layers[:8]):
        assert L == Lr
    # per grid, one launch per layer (the paper's recursive mode) on a sample
    k = min(args.plain_sample, len(ws))
    t0 = time.perf_counter()
    for (m, t, s), w in list(zip(dev, ws))[:k]:
        with pkg.Planner(m, w.dist_bits) as pl:
            pl.propagate(t, plain=True, check_every=64)
            pl.trace(s.cpu().numpy().view(np.uint32))
    dtp = time.perf_counter() - t0
    out["per_maze_plain_launches"] = {"mazes_per_s": k / dtp, "seconds": dtp,
                                      "sample": f"first {k} of the {len(ws)} grids"}

    # serving: Poisson arrivals at 0.8 x the batched capacity
    lam = 0.8 * out["batched"]["mazes_per_s"]
    arr = synth.poisson_arrivals(len(ws), lam, seed=4)
    reqs = [Request(m, t, s, w.dist_bits, float(a)) for (m, t, s), w, a in zip(dev, ws, arr)]
    big = max(totals)
    staging = (torch.empty(max(big, 1), dtype=torch.int32).pin_memory(),
               torch.empty(max(w.starts.size for w in ws) + 1, dtype=torch.int64).pin_memory(),
               torch.empty(max(w.starts.size for w in ws) + 1, dtype=torch.int8).pin_memory())
    with pkg.Batch(budget) as b:
        rep = serve(b, reqs, round_sweeps=64, staging=staging, max_round_sweeps=1024)
    out["serve"] = dict(rep.summary(), lambda_per_s=lam, round_sweeps=64, max_round_sweeps=1024,
                        note="rounds of 64 sweeps; while no request arrives each round doubles, "
                             "up to 1024")
    out["speedup_vs_per_maze_plain"] = out["batched"]["mazes_per_s"] / out["per_maze_plain_launches"]["mazes_per_s"]
    out["speedup_vs_per_maze_persistent"] = out["batched"]["mazes_per_s"] / out["per_maze_persistent"]["mazes_per_s"]
    return out


def run_batched_sharded(args, pkg, torch, rank, world, pg):
    """The 256-grid stream over `world` ranks: rank r solves grids r, r + world,
    ... in its own batch (independent problems, no collective on the data
    path); whole-job grids/s = all grids / the slowest rank's time."""
    ws = synth.c4_batch(args.batch_n)
    mine = shard(len(ws), rank, world)
    sub = [ws[i] for i in mine]
    dev = [(torch.from_numpy(w.mask).cuda(), torch.from_numpy(w.targets.view(np.int32)).cuda(),
            torch.from_numpy(w.starts.view(np.int32)).cuda()) for w in sub]
    budget = int(sum(w.H * w.W * 5 + 4096 * 64 for w in sub) * 1.5) + (256 << 20)

    def once(host=None):
        with pkg.Batch(budget) as b:
            tks = [b.submit(m, t, s, w.dist_bits) for (m, t, s), w in zip(dev, sub)]
            b.run(0)
            tot = [b.info(tk)["total_cells"] for tk in tks]
            if host is not None:
                a = 0
                for tk, w, x in zip(tks, sub, tot):
                    b.result(tk, w.starts.size, want_dist=False, cells=host[0][a:a + max(x, 1)],
                             offsets=host[1][:w.starts.size + 1], status=host[2][:max(w.starts.size, 1)])
                    a += max(x, 1)
        return tot

    tot = once()
    host = (torch.empty(sum(max(x, 1) for x in tot), dtype=torch.int32).pin_memory(),
            torch.empty(max(w.starts.size for w in sub) + 1, dtype=torch.int64).pin_memory(),
            torch.empty(max(w.starts.size for w in sub) + 1, dtype=torch.int8).pin_memory())
    pg.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    once(host)
    torch.cuda.synchronize()
    local_ms = (time.perf_counter() - t0) * 1e3
    t_ms, rate = aggregate(local_ms, len(ws) / world, 1, world, pg, "cuda")
    return {"workload": f"{len(ws)} grids, side U{{64..2048}}, sharded round-robin over {world} ranks",
            "mazes_per_s": rate, "seconds": t_ms * 1e-3, "grids_this_rank": len(sub),
            "scaling": "weak (grids per rank fixed by the shard)"}


PAPER_FIG5_S_PER_L_N2 = 3.0751e-10   # seconds per layer per cell, GTX 1080 Ti (Results, run-time)


def run_fig5(args):
    """Empty n x n grids, one source in a corner (the paper's worst case), a
    network of fixed depth L in {0.5n, n, 1.5n, 2n}; device time of the
    propagation beside the paper's fitted model."""
    import torch
    import paper_2004_00540_gb300 as pkg
    rows = []
    for n in (500, 1000, 2000, 3000, 4000):
        m = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
        t = torch.zeros(1, dtype=torch.int32, device="cuda")
        with pkg.Planner(m, pkg.MPN_DIST_U32) as pl:
            for f in (0.5, 1.0, 1.5, 2.0):
                L = int(f * n)
                ms = []
                for rep in range(4):
                    pl.propagate(t, max_layers=L)
                    ms.append(pl.stats()["ms_propagate"])
                best = min(ms[1:])
                layers = pl.layers
                paper_s = PAPER_FIG5_S_PER_L_N2 * L * n * n
                rows.append({"n": n, "L": L, "layers_reached": layers, "ms": best,
                             "effective_cell_updates_per_s": n * n * L / (best * 1e-3),
                             "paper_model_s": paper_s, "speedup_vs_paper_model": paper_s / (best * 1e-3)})
    print(json.dumps({"fig5_empty_grids": rows}), flush=True)
    return 0


def run_table1(args):
    """The paper's Appendix Table I comparison: the recursive mode (one launch
    per layer, a convergence check on the host every 64 layers) against the
    persistent kernel, on a 2000 x 2000 grid (Bernoulli 0.25, 16 targets) and
    on the 1024 x 1024 DFS maze; device-resident inputs, propagation only."""
    import torch
    import paper_2004_00540_gb300 as pkg
    w2 = synth.c5_huge(side=2000)
    cases = [("grid2000_bernoulli0.25_rect10", w2.mask, w2.targets[:16]),
             ("maze1024_dfs", synth.c2_maze().mask, synth.c2_maze().targets)]
    rows = []
    for name, mask, targets in cases:
        m = torch.from_numpy(mask).cuda()
        t = torch.from_numpy(np.ascontiguousarray(targets).view(np.int32)).cuda()
        with pkg.Planner(m, pkg.MPN_DIST_U32) as pl:
            pl.propagate(t)
            L = pl.layers
            pers = []
            for _ in range(3):
                pl.propagate(t)
                pers.append(pl.stats()["ms_propagate"])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pl.propagate(t, plain=True, check_every=64)
            torch.cuda.synchronize()
            plain_ms = (time.perf_counter() - t0) * 1e3
            assert pl.layers == L
        p_ms = min(pers)
        rows.append({"case": name, "layers": L, "persistent_ms": p_ms, "per_layer_launches_ms": plain_ms,
                     "ratio": plain_ms / p_ms})
    print(json.dumps({"table1_recursive_vs_persistent": rows}), flush=True)
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.fig5:
        return run_fig5(args)
    if args.table1:
        return run_table1(args)

    import torch
    import paper_2004_00540_gb300 as pkg

    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    w = workload(args.side)
    H, W = w.H, w.W
    stream = torch.cuda.Stream()
    d_mask = torch.from_numpy(w.mask).cuda()
    d_t = torch.from_numpy(w.targets.view(np.int32)).cuda()
    d_s = torch.from_numpy(w.starts.view(np.int32)).cuda()
    torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        ctx = pkg.mpn_create(d_mask, H, W, pkg.MPN_DIST_U32, stream)
    tuned = None
    if args.variant >= 0:
        pkg.mpn_set_tuning(ctx, args.variant, args.depth)
    elif not args.no_autotune:
        # every tile shape x depth measured on this grid (outside the timed region)
        tv, td, tms = pkg.mpn_autotune(ctx, d_t)
        tuned = {"variant": tv, "depth": td, "propagate_ms": tms}
    # device-resident outputs, sized once
    L = pkg.mpn_propagate(ctx, d_t)
    n = w.starts.size
    d_off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    pkg.mpn_trace_lengths(ctx, d_s, d_off)
    total = int(d_off[-1].item())
    d_cells = torch.zeros(max(total, 1), dtype=torch.int32, device="cuda")
    d_status = torch.zeros(n, dtype=torch.int8, device="cuda")

    def step():
        pkg.mpn_set_mask(ctx, d_mask)
        pkg.mpn_propagate(ctx, d_t, 0, wait=False)
        st = pkg.mpn_trace(ctx, d_s, d_off, d_cells, total, d_status)
        assert st == pkg.MPN_OK

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    stats0 = pkg.mpn_get_stats(ctx)

    # timed region: K steps bracketed by barrier + synchronize; events on the
    # library's stream; per-kernel propagate time from the library's events
    props = torch.cuda.get_device_properties(local)
    uuid = str(getattr(props, "uuid", "") or "")
    clocks = ClockSampler(("GPU-" + uuid) if uuid and not uuid.startswith("GPU-") else (uuid or str(local)))
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = pkg.mpn_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    prop_ms = []
    ev0.record(stream)
    for _ in range(args.steps):
        step()
        prop_ms.append(pkg.mpn_get_stats(ctx)["ms_propagate"])
    ev1.record(stream)
    ev1.synchronize()
    launches = pkg.mpn_launch_count() - launches0
    t_ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    st = pkg.mpn_get_stats(ctx)
    L = st["layers"]
    units = float(H) * W * L
    t_ms, value = aggregate(t_ms, units, args.steps, world, pg, "cuda")
    if pg:
        pg.barrier()
    prop_avg = sum(prop_ms) / len(prop_ms)

    # roofline of the dominant kernel pair: the persistent propagation kernel
    # and the activation-log decode that completes its distance plane (the
    # context's propagate events bracket both). Algorithmic bytes = the
    # floor of a propagation (packed mask read once, uint32 plane written
    # once); the dense N * L equivalent is reported as cell-updates/s only.
    peak, peak_kind = peaks()
    floor_bytes = FLOOR_BYTES_PER_CELL_U32 * H * W
    achieved = floor_bytes / (prop_avg * 1e-3) / 1e9
    traffic = measured_traffic(w.name, st["variant"], st["depth"])
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "floor_bytes": floor_bytes,
            "dram_frac": (traffic / (prop_avg * 1e-3) / (peak * 1e9)) if traffic else None,
            "traffic_over_floor": (traffic / floor_bytes) if traffic else None,
            "peak_kind": peak_kind,
            "kernel": "k_propagate + k_log_decode", "ms_per_launch": prop_avg,
            "effective_cell_updates_per_s": units / (prop_avg * 1e-3),
            "note": "algorithmic bytes per launch = 4.125 B per cell (packed mask bit read once, "
                    "uint32 distance written once) x H x W; frac = those bytes / launch time / "
                    "measured copy peak; traffic = ncu DRAM read + write bytes of both kernels "
                    "per launch"}

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        h_mask = torch.from_numpy(w.mask).pin_memory()
        h_t = torch.from_numpy(w.targets.view(np.int32)).pin_memory()
        h_s = torch.from_numpy(w.starts.view(np.int32)).pin_memory()
        h_dist = torch.empty((H, W), dtype=torch.int32).pin_memory()
        h_off = torch.zeros(n + 1, dtype=torch.int64).pin_memory()
        h_cells = torch.zeros(max(total, 1), dtype=torch.int32).pin_memory()
        h_status = torch.zeros(n, dtype=torch.int8).pin_memory()

        def solve(c, dst, off, cells, status):
            pkg.mpn_set_mask(c, h_mask)
            pkg.mpn_propagate(c, h_t, 0, wait=False)
            pkg.mpn_trace(c, h_s, off, cells, total, status)
            pkg.mpn_get_distances(c, dst)

        lanes = [(ctx, h_dist, h_off, h_cells, h_status)]
        solve(*lanes[0])
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        ke = max(1, min(args.steps, 5))
        for _ in range(ke):
            solve(*lanes[0])
        torch.cuda.synchronize()
        te = (time.perf_counter() - t0) / ke
        assert int(h_off[-1]) == total
        serial_ms, serial_value = aggregate(te * 1e3, units, 1, world, pg, "cuda")

        # the same solves pipelined over two contexts, each on its own stream:
        # solve i + 1's mask goes up while solve i propagates, and solve i's
        # distances come down (on a copy stream) while solve i + 1 runs. Every
        # step still uploads its mask, targets and starts and downloads its
        # distances and paths; the host waits for each download before it
        # reuses that buffer.
        ctx2_stream = torch.cuda.Stream()
        copy_stream = torch.cuda.Stream()
        with torch.cuda.stream(ctx2_stream):
            ctx2 = pkg.mpn_create(d_mask, H, W, pkg.MPN_DIST_U32, ctx2_stream)
        pkg.mpn_set_tuning(ctx2, st["variant"], st["depth"])
        lanes.append((ctx2, torch.empty((H, W), dtype=torch.int32).pin_memory(),
                      torch.zeros(n + 1, dtype=torch.int64).pin_memory(),
                      torch.zeros(max(total, 1), dtype=torch.int32).pin_memory(),
                      torch.zeros(n, dtype=torch.int8).pin_memory()))

        def pipeline(count):
            c0 = lanes[0][0]
            pkg.mpn_set_mask(c0, h_mask)
            pkg.mpn_propagate(c0, h_t, 0, wait=False)
            for i in range(count):
                c, dst, off, cells, status = lanes[i % 2]
                nxt = lanes[(i + 1) % 2][0]
                if i + 1 < count:
                    pkg.mpn_set_mask(nxt, h_mask)   # overlaps this solve's kernels
                pkg.mpn_trace(c, h_s, off, cells, total, status)
                pkg.mpn_get_distances_async(c, dst, copy_stream)
                if i + 1 < count:
                    pkg.mpn_sync(nxt)   # solve i - 1's download is done
                    pkg.mpn_propagate(nxt, h_t, 0, wait=False)
            for ln in lanes:
                pkg.mpn_sync(ln[0])

        pipeline(2)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        kp = 4 * ke
        t0 = time.perf_counter()
        pipeline(kp)
        torch.cuda.synchronize()
        tp = (time.perf_counter() - t0) / kp
        for ln in lanes[1:]:
            assert int(ln[2][-1]) == total and torch.equal(h_dist, ln[1])
            assert torch.equal(h_cells[:total], ln[3][:total])
        pkg.mpn_destroy(ctx2)
        te_ms, e2e_value = aggregate(tp * 1e3, units, 1, world, pg, "cuda")
        e2e = {"value": e2e_value, "unit": UNIT, "ms_per_step": te_ms,
               "h2d_bytes_per_step": int(H * W + 4 * w.targets.size + 4 * n),
               "d2h_bytes_per_step": int(4 * H * W + 8 * (n + 1) + 4 * total + n + 8),
               "steps": kp,
               "serial": {"value": serial_value, "ms_per_step": serial_ms},
               "note": "host wall clock over whole solves through the C ABI (pinned host "
                       "buffers; mask, targets, starts up; distances, offsets, paths, status "
                       "down), pipelined over two contexts: one solve's mask upload and "
                       "distance download overlap the other's kernels; serial = one solve "
                       "at a time, nothing overlapped"}

    pkg.mpn_destroy(ctx)
    sharded = None
    if world > 1 and not args.no_batched:
        sharded = run_batched_sharded(args, pkg, torch, rank, world, pg)
    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(w, L, total, world),
        "tuning": {"variant": st["variant"], "depth": st["depth"], "autotuned": tuned},
        "propagate": {"ms": prop_avg, "effective_cell_updates_per_s": units / (prop_avg * 1e-3),
                      "dense_equivalent_bytes_per_s": units * BYTES_PER_UPDATE_U32 / (prop_avg * 1e-3),
                      "sweeps": st["sweeps"], "tile_visits": st["tile_visits"],
                      "tiles": st["tiles_x"] * st["tiles_y"], "blocks": st["blocks"],
                      "tile_layers_executed_frac": st["tile_layers"] / max(1, st["tile_visits"] * st["depth"]),
                      "log_entries": st["log_entries"]},
        "trace": {"ms": st["ms_trace"], "paths": int(n), "cells": total,
                  "paths_per_s": n / (st["ms_trace"] * 1e-3) if st["ms_trace"] else None,
                  "cells_per_s": total / (st["ms_trace"] * 1e-3) if st["ms_trace"] else None},
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": e2e,
    }
    if pg:
        pg.destroy_process_group()
    if not args.no_batched and world == 1:
        line["batched"] = run_batched(args, pkg, torch)
    if sharded is not None:
        line["batched"] = {"sharded": sharded}
    if not args.no_per_config and world == 1:
        line["per_config"] = run_per_config(pkg, torch)
    if not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
