"""Continuous-batching request loop over the batched engine (include/mpn.h,
mpn_batch_*).

Requests (a grid, its targets and starts) arrive over time. The loop admits
waiting requests in arrival order while the batch's device arena has room
(admission by device memory), runs one round -- one persistent launch that
advances every admitted grid for a bounded number of sweeps -- collects the
grids that finished (their paths are downloaded as the response) and
releases them, so that arrivals during a round join at the next one. All
GPU work runs in the library; this module only schedules and keeps time.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from .mpn import Batch, MPN_BATCH_DONE, MPN_BATCH_PENDING


@dataclass
class Request:
    mask: np.ndarray
    targets: np.ndarray
    starts: np.ndarray
    dist_bits: int = 0
    arrival: float = 0.0          # seconds after the start of the run


@dataclass
class ServeReport:
    latencies: list = field(default_factory=list)   # seconds, per request, arrival -> response
    makespan: float = 0.0
    rounds: int = 0
    refused_admissions: int = 0                      # submit attempts that did not fit yet
    results: dict = field(default_factory=dict)      # request index -> Paths (if kept)
    failed: list = field(default_factory=list)
    round_sweeps: list = field(default_factory=list)  # sweep budget of each round

    def summary(self) -> dict:
        lat = np.asarray(self.latencies) * 1e3
        n = len(self.latencies)
        return {
            "requests": n,
            "makespan_s": self.makespan,
            "mazes_per_s": n / self.makespan if self.makespan > 0 else None,
            "p50_ms": float(np.percentile(lat, 50)) if n else None,
            "p99_ms": float(np.percentile(lat, 99)) if n else None,
            "mean_ms": float(lat.mean()) if n else None,
            "rounds": self.rounds,
            "refused_admissions": self.refused_admissions,
            "failed": len(self.failed),
        }


def _count(a) -> int:
    """Element count of a numpy array or a torch tensor."""
    return int(a.numel()) if hasattr(a, "numel") else int(np.asarray(a).size)


def _own(a):
    """A host numpy copy of an array or tensor view."""
    return np.array(a.numpy() if hasattr(a, "numpy") else a, copy=True)


def serve(batch: Batch, requests: list, round_sweeps: int = 64, keep_results: bool = False,
          clock=time.perf_counter, staging=None, max_round_sweeps: int = 0) -> ServeReport:
    """Run every request through the batch as it arrives; returns latencies.
    staging: optional (cells, offsets, status) host buffers (page-locked is
    fastest), each large enough for any one response; every response is
    downloaded into them (and copied out when kept) instead of into freshly
    allocated arrays. max_round_sweeps > round_sweeps: while no request has
    arrived since the last round, each round runs twice as many sweeps as the
    one before, up to max_round_sweeps (fewer rounds, so less time between
    them, for the grids that need many sweeps); an arrival brings the rounds
    back to round_sweeps, so that it joins soon."""
    rep = ServeReport()
    cur = round_sweeps
    order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
    waiting = collections.deque()
    in_flight = {}                 # ticket -> request index
    nxt = 0
    t0 = clock()
    while nxt < len(order) or waiting or in_flight:
        now = clock() - t0
        arrived = False
        while nxt < len(order) and requests[order[nxt]].arrival <= now:
            waiting.append(order[nxt])
            nxt += 1
            arrived = True
        while waiting:
            r = requests[waiting[0]]
            tk = batch.submit(r.mask, r.targets, r.starts, r.dist_bits)
            if tk is None:
                rep.refused_admissions += 1
                break
            in_flight[tk] = waiting.popleft()
        if in_flight:
            if arrived or waiting or max_round_sweeps <= round_sweeps:
                cur = round_sweeps
            batch.run(cur)
            rep.rounds += 1
            rep.round_sweeps.append(cur)
            cur = min(2 * cur, max(max_round_sweeps, round_sweeps))
            for tk in list(in_flight):
                st = batch.poll(tk)
                if st == MPN_BATCH_PENDING:
                    continue
                i = in_flight.pop(tk)
                if st == MPN_BATCH_DONE:
                    n = _count(requests[i].starts)
                    if staging is not None:
                        _, paths, _ = batch.result(tk, n, want_dist=False, cells=staging[0],
                                                   offsets=staging[1], status=staging[2])
                        if keep_results:
                            paths = type(paths)(_own(paths.offsets), _own(paths.cells),
                                                _own(paths.status))
                    else:
                        _, paths, _ = batch.result(tk, n, want_dist=False)
                    if keep_results:
                        rep.results[i] = paths
                else:
                    rep.failed.append(i)
                batch.release(tk)
                rep.latencies.append(clock() - t0 - requests[i].arrival)
        elif nxt < len(order):
            wait = requests[order[nxt]].arrival - (clock() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.05))
    rep.makespan = clock() - t0
    return rep

