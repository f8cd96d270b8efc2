"""The continuous-batching request loop (paper_2004_00540_gb300/serve.py)
against a fake batch engine on the CPU: admission in arrival order while the
arena has room, arrivals joining at the next round, completions released and
timed, failures reported, and nothing left behind."""
import numpy as np

from paper_2004_00540_gb300 import serve as sv
from paper_2004_00540_gb300.mpn import MPN_BATCH_DONE, MPN_BATCH_FAILED, MPN_BATCH_PENDING


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBatch:
    """Holds at most `slots` grids; a grid needs `work` sweeps (its first
    mask value) and fails if that value is negative. Each run advances every
    held grid by the round's sweeps and moves the clock by 1 ms."""

    def __init__(self, slots, clock):
        self.slots, self.clock = slots, clock
        self.held = {}
        self.failing = set()
        self.next_ticket = 1
        self.submitted = []
        self.released = []

    def submit(self, mask, targets, starts, dist_bits=0):
        if len(self.held) >= self.slots:
            return None
        tk = self.next_ticket
        self.next_ticket += 1
        work = int(mask.reshape(-1)[0])
        if work < 0:
            self.failing.add(tk)
        self.held[tk] = abs(work)
        self.submitted.append(tk)
        return tk

    def run(self, sweeps):
        self.clock.t += 1e-3
        for tk in self.held:
            self.held[tk] -= sweeps

    def poll(self, tk):
        if tk in self.failing:
            return MPN_BATCH_FAILED
        return MPN_BATCH_DONE if self.held[tk] <= 0 else MPN_BATCH_PENDING

    def result(self, tk, n, want_dist=False):
        return None, ("paths", tk, n), None

    def release(self, tk):
        self.released.append(tk)
        del self.held[tk]


def req(work, arrival, n_starts=3):
    m = np.zeros((2, 2), np.int64)
    m[0, 0] = work
    return sv.Request(m, np.array([1], np.uint32), np.arange(n_starts, dtype=np.uint32), 0, arrival)


def test_admission_rounds_and_latencies():
    clock = FakeClock()
    b = FakeBatch(slots=2, clock=clock)
    reqs = [req(64, 0.0), req(128, 0.0), req(64, 0.0), req(64, 0.0)]
    rep = sv.serve(b, reqs, round_sweeps=64, keep_results=True, clock=clock)
    # two fit at a time: the third and fourth waited for room
    assert rep.refused_admissions >= 1
    assert sorted(rep.results) == [0, 1, 2, 3]
    assert len(rep.latencies) == 4 and all(x > 0 for x in rep.latencies)
    assert not b.held and sorted(b.released) == sorted(b.submitted)
    assert rep.results[2][2] == 3   # the start count reaches the result call
    s = rep.summary()
    assert s["requests"] == 4 and s["failed"] == 0 and s["rounds"] == rep.rounds
    assert s["p50_ms"] <= s["p99_ms"]


def test_arrivals_join_at_the_next_round():
    clock = FakeClock()
    b = FakeBatch(slots=8, clock=clock)
    # a long grid first; a short one arrives while it runs and finishes first
    reqs = [req(640, 0.0), req(64, 0.0025)]
    rep = sv.serve(b, reqs, round_sweeps=64, keep_results=True, clock=clock)
    assert rep.refused_admissions == 0
    assert b.submitted == [1, 2]                 # arrival order
    assert b.released.index(2) < b.released.index(1)
    assert rep.latencies[0] < rep.latencies[1]   # short request answered first
    assert rep.rounds == 10


def test_failures_are_reported_and_released():
    clock = FakeClock()
    b = FakeBatch(slots=4, clock=clock)
    reqs = [req(64, 0.0), req(-64, 0.0)]
    rep = sv.serve(b, reqs, round_sweeps=64, clock=clock)
    assert rep.failed == [1]
    assert not b.held
    assert rep.summary()["failed"] == 1


def test_rounds_grow_while_nothing_arrives():
    clock = FakeClock()
    b = FakeBatch(slots=4, clock=clock)
    reqs = [req(2000, 0.0), req(64, 0.0035)]
    rep = sv.serve(b, reqs, round_sweeps=64, clock=clock, max_round_sweeps=512)
    # the long grid alone: 64, 128, 256, 512 sweeps; the second request arrives
    # during the 512-sweep round and the next round is short again
    assert rep.round_sweeps[:6] == [64, 128, 256, 512, 64, 128]
    assert max(rep.round_sweeps) == 512
    assert sum(rep.round_sweeps) >= 2000
    assert sorted(b.released) == sorted(b.submitted)
    # the late request finished in the round right after it arrived
    assert abs(rep.latencies[0] - 0.0015) < 1e-9


def test_fixed_rounds_by_default():
    clock = FakeClock()
    b = FakeBatch(slots=4, clock=clock)
    rep = sv.serve(b, [req(1000, 0.0)], round_sweeps=64, clock=clock)
    assert rep.round_sweeps == [64] * 16
