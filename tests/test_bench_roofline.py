"""The bench's roofline record on CPU: the ALU peaks from unit counts and
clocks, the dominant evaluation kernel's fraction from its live time, and the
profiled DRAM traffic chosen by the Gaussian state the step ran on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_alu_peaks_from_unit_counts():
    # forward: 3 FP32 + 1 ex2 per pair, the MUFU (32 per SM per clock) binds
    assert bench.alu_peak_pairs("render_fwd") == pytest.approx(148 * 32 * 2032e6)
    # backward: 5 FP32 + 1 ex2 per pair, the FP32 lanes (128 per SM per clock) bind
    assert bench.alu_peak_pairs("render_bwd") == pytest.approx(148 * 128 / 5 * 2032e6)


@pytest.mark.parametrize("state", ["initial", "fitted"])
def test_roofline_takes_the_slower_kernel_and_its_traffic(state):
    pairs = 9.2e8
    # stage -> (total ms over the steps, launches)
    stages = {"render_fwd": (2.2, 10), "render_bwd": (2.7, 10), "chain": (0.7, 10)}
    traffic = bench.PROFILED_TRAFFIC[state]
    r = bench.roofline(stages, pairs, traffic=traffic)
    assert r["kernel"] == "render_bwd"
    assert r["ms_per_launch"] == pytest.approx(0.27)
    achieved = pairs / 0.27e-3
    assert r["achieved"] == pytest.approx(achieved / 1e9)
    assert r["frac"] == pytest.approx(achieved / bench.alu_peak_pairs("render_bwd"))
    assert r["traffic"] == traffic["render_bwd"]
    fwd = r["other"]["render_fwd"]
    assert fwd["ms"] == pytest.approx(0.22)
    assert fwd["frac"] == pytest.approx(pairs / 0.22e-3 / bench.alu_peak_pairs("render_fwd"))
    assert fwd["traffic"] == traffic["render_fwd"]  # None once the kernel changed since its capture


def test_roofline_without_a_capture_reports_no_traffic():
    stages = {"render_fwd": (3.0, 10), "render_bwd": (2.0, 10)}
    r = bench.roofline(stages, 1e9, traffic=bench.PROFILED_TRAFFIC.get("loaded"))
    assert r["kernel"] == "render_fwd"
    assert r["traffic"] is None and r["other"]["render_bwd"]["traffic"] is None
