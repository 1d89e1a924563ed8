"""bench.py's host arithmetic (no GPU): the roofline of a kernel launch is
the slower of its algorithmic flops at the form's pipe peak and its
algorithmic bytes at the measured bandwidth, and its fraction is that bound's
time over the measured time."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.fixture(autouse=True)
def fixed_peaks(monkeypatch):
    monkeypatch.setitem(bench.PEAK_TFLOPS, "fp32", 80.0)
    monkeypatch.setitem(bench.PEAK_TFLOPS, "fp64", 1.25)


def test_edge_flops_are_the_methods_per_step_counts():
    """700 flops per Gauss point and layer for the gas-kinetic solution (two
    points, two layers) plus both cells' polynomials (value and gradient of
    six variables, 27 multiply-adds each) at the two points."""
    assert bench.WORK_PER_UNIT["edge_fused"][0] == 2 * 2 * 700 + 2 * (2 * 2) * 6 * 27 == 4096
    assert bench.recon_flops(0.0) == 2 * (918 + 180 + 600)
    assert bench.recon_flops(1.0) == 2 * 918


def test_fused_edge_kernel_takes_the_slower_of_its_limits():
    """The fused edge kernel's flops and bytes per edge are nearly balanced
    (4096 flops at the FP32 peak against 366 bytes at the bandwidth): its
    fraction is the slower limit's time over the launch time."""
    fl, by = bench.WORK_PER_UNIT["edge_fused"]
    units, ms = 3_000_000, 0.6
    for hbm in (6800.0, 9000.0):
        r = bench.roofline("fp32_learned", "edge_fused", units, ms, hbm)
        t_alu, t_hbm = fl * units / 80e12, by * units / (hbm * 1e9)
        assert r["kernel"] == "k_edgef"
        assert r["frac"] == pytest.approx(max(t_alu, t_hbm) / (ms * 1e-3))
        assert r["bound"] == ("hbm" if t_hbm > t_alu else "alu")
    assert r["pipe"] == "fp32" and r["achieved"] == pytest.approx(fl * units / (ms * 1e-3) / 1e12)


def test_fp64_form_is_bound_by_the_fp64_pipe():
    fl, _ = bench.WORK_PER_UNIT["edge"]
    units, ms, hbm = 3_000_000, 20.0, 6800.0
    r = bench.roofline("fp64", "edge", units, ms, hbm)
    assert r["bound"] == "alu" and r["pipe"] == "fp64" and r["peak"] == 1.25
    assert r["frac"] == pytest.approx(fl * units / (ms * 1e-3) / 1.25e12)


def test_reconstruction_is_bound_by_its_bytes():
    """A cell with the nonlinear weights also reads its P1 rows and
    smoothness forms (75 words): 1069 bytes per smooth cell, 1369 per
    troubled one."""
    assert bench.recon_bytes(1.0) == bench.WORK_PER_UNIT["recon"][1] == 1069
    assert bench.recon_bytes(0.0) == 1069 + 300
    units, ms, hbm = 2_000_000, 0.55, 6800.0
    r = bench.roofline("fp32", "recon", units, ms, hbm, smooth_fraction=0.9)
    by = 1069 + 0.1 * 300
    assert r["bound"] == "hbm" and r["kernel"] == "k_recon" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(by * units / (ms * 1e-3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / hbm)


def test_every_timed_kernel_has_work_figures():
    for k in ("recon", "gate", "iface", "edge", "edge_fused", "update"):
        fl, by = bench.WORK_PER_UNIT[k]
        assert fl > 0 and by > 0
        assert bench.EXECUTED_FP32_PER_UNIT[k] > 0


def test_workload_samples_keep_the_workload():
    """The CPU baseline's and the reference arm's bounded samples are the
    headline workload at fewer squares per side."""
    p = bench.make_workload("large", bench.SAMPLE_SCALE["large"])
    assert (p.mesh.nx, p.mesh.ny) == (128, 16) and p.chi == 0.97
    assert p.mesh.domain == (0.0, 8.0, 0.0, 1.0)
    assert bench.n_edges(p) == (3 * p.mesh.n_tri + 2 * (128 + 16)) // 2
