"""bench.py reports the DRAM traffic and FP32 work recorded in the committed ncu summary of the
dominant kernel only for the grid it was captured on and only while the kernel's sources hash to
the value recorded with them."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _recorded_hash():
    with open(os.path.join(ROOT, bench.HOT_KERNEL_PROFILE)) as f:
        for line in f:
            if line.startswith("source_hash:"):
                return line.split(":", 1)[1].strip()
    return None


def test_recorded_traffic_is_reported_for_the_captured_grid_only(monkeypatch):
    monkeypatch.setattr(bench, "hot_kernel_hash", _recorded_hash)
    assert bench.recorded_traffic((2048, 2048)) == 284.0e6
    assert bench.recorded_profile("fp32_flops_per_launch", (2048, 2048)) > 0
    assert bench.recorded_traffic((128, 128)) is None
    assert bench.recorded_traffic((256, 256, 256)) is None


def test_recorded_traffic_is_dropped_when_the_sources_change(monkeypatch):
    monkeypatch.setattr(bench, "hot_kernel_hash", lambda: "0" * 16)
    assert bench.recorded_traffic((2048, 2048)) is None
