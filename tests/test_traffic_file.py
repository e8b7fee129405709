"""The committed DRAM counters that bench.py reports as the roofline "traffic"
field: well formed, one entry per kernel identity, bytes per point within a few
percent of the kernel's algorithmic bytes (a figure far above them would mean
re-reads; far below, a counter of the wrong kernel)."""

import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# algorithmic bytes per point of each step kind (FP32 fields, 2-byte snapshot levels)
ALGORITHMIC = {"plain": 16, "snap_fp32": 20, "snap_bf16": 18, "snap_fp16": 18,
               "grad_fp32": 28, "grad_bf16": 26, "grad_fp16": 26}


def test_traffic_file_is_well_formed():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        t = json.load(fh)
    assert t["points_per_launch"] > 0 and t["captures"]
    for c in t["captures"]:
        assert "--clock-control none" in c["command"] and c["plain_run"]
    assert t["kernels"]
    for key, e in t["kernels"].items():
        assert len(key) == 16 and int(key, 16) >= 0
        alg = ALGORITHMIC[e["step"]]
        assert e["dram_bytes_per_point"] == pytest.approx(
            (e["dram_read_bytes"] + e["dram_write_bytes"]) / t["points_per_launch"], rel=1e-3)
        assert 0.85 * alg <= e["dram_bytes_per_point"] <= 1.05 * alg, (key, e)


def test_bench_reads_the_traffic_file():
    import bench
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        key, e = next(iter(json.load(fh)["kernels"].items()))
    assert bench.measured_traffic(key, 1000) == pytest.approx(1000 * e["dram_bytes_per_point"])
    assert bench.measured_traffic("0" * 16, 1000) is None
