"""bench.py's host arithmetic (no GPU): the roofline of a kernel launch is
the slowest of its FP32 work, FP64 work and algorithmic bytes at the peaks,
and its fraction is that bound's time over the measured time."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.fixture(autouse=True)
def fixed_peaks(monkeypatch):
    monkeypatch.setitem(bench.PEAK_TFLOPS, "fp32", 80.0)
    monkeypatch.setitem(bench.PEAK_TFLOPS, "fp64", 1.25)


def test_fused_edge_kernel_is_bound_by_fp32_work():
    f32, f64, by = bench.WORK_PER_UNIT["fp32"]["edge_fused"]
    units, ms, hbm = 3_000_000, 0.6, 6800.0
    r = bench.roofline("fp32", "edge_fused", units, ms, hbm)
    assert r["bound"] == "alu" and r["pipe"] == "fp32" and r["kernel"] == "k_edgef"
    assert r["achieved"] == pytest.approx(f32 * units / (ms * 1e-3) / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 80.0)
    assert f32 * units / 80e12 > by * units / (hbm * 1e9)          # the FP32 time is the longest


def test_reconstruction_is_bound_by_its_bytes():
    f32, f64, by = bench.WORK_PER_UNIT["fp32"]["recon"]
    units, ms, hbm = 2_000_000, 0.55, 6800.0
    r = bench.roofline("fp32", "recon", units, ms, hbm)
    assert r["bound"] == "hbm" and r["kernel"] == "k_recon" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(by * units / (ms * 1e-3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / hbm)


def test_every_timed_kernel_has_work_and_traffic_figures():
    for k in ("recon", "gate", "iface", "edge", "edge_fused", "update"):
        f32, f64, by = bench.WORK_PER_UNIT["fp32"][k]
        assert f32 > 0 and by > 0 and f64 >= 0
    for k in ("recon", "gate", "edge_fused", "update"):
        assert bench.TRAFFIC_PER_UNIT["fp32"][k] > 0
