"""Host logic of bench.py that needs no GPU: the committed DRAM-traffic figure
is used only while the kernel sources, the workload and the tiling it was
captured on match the run."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture()
def bench():
    return load_bench()


def write_capture(path, **kw):
    with open(path, "w") as f:
        json.dump(kw, f)


def test_committed_capture_is_consistent(bench):
    # (a capture older than the kernel sources is allowed: bench.py then
    # reports no traffic figure, see the next test)
    with open(bench.TRAFFIC_FILE) as f:
        t = json.load(f)
    assert len(t["source_sha256"]) == 64
    assert t["dram_bytes_per_launch"] == pytest.approx(t["dram_bytes_read"] + t["dram_bytes_write"])
    per = t["per_kernel"]
    assert sum(k["dram_bytes_read"] for k in per.values()) == pytest.approx(t["dram_bytes_read"])


def test_traffic_needs_same_sources_workload_and_tiling(bench, tmp_path, monkeypatch):
    f = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    h = bench.kernel_source_hash()
    write_capture(f, source_sha256=h, workload="w", variant=0, depth=24, dram_bytes_per_launch=5e9)
    assert bench.measured_traffic("w", 0, 24) == 5e9
    assert bench.measured_traffic("other", 0, 24) is None
    assert bench.measured_traffic("w", 1, 24) is None
    assert bench.measured_traffic("w", 0, 16) is None
    write_capture(f, source_sha256="0" * 64, workload="w", variant=0, depth=24, dram_bytes_per_launch=5e9)
    assert bench.measured_traffic("w", 0, 24) is None
    f.unlink()
    assert bench.measured_traffic("w", 0, 24) is None


def test_source_hash_covers_the_propagation_kernels(bench):
    h1 = bench.kernel_source_hash()
    assert len(h1) == 64 and h1 == bench.kernel_source_hash()
