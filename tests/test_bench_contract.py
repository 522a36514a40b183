"""Host-side parts of bench.py (no GPU): the roofline object of the dominant kernel
and the launch count of the timed region follow the contract's definitions."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_roofline_of_the_dominant_kernel():
    # (mean ms per launch, launches, algorithmic bytes per launch, flops, iterations)
    stats = {"iterate": (2.87, 2, 1.790e9, 3.4e8, 800), "sa_msys": (2.75, 2, 2.87e10, 1e9, 2),
             "refresh": (0.67, 2, 1.64e9, 1.6e9, 2)}
    r = bench.roofline(stats, {"hbm_gbs": 6788.3})
    assert r["kernel"] == "iterate" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 1.790e9 / 2.87e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 6788.3) < 1e-12
    # ncu traffic (228.7 MB per 50 iterations) scaled to the iterations of one launch
    # (400 here)
    assert abs(r["traffic"] - bench.PROFILED_TRAFFIC["iterate"](400)) < 1.0
    assert abs(r["traffic"] - 8 * 228.7e6) < 1e3


def test_roofline_falls_back_without_measured_peaks():
    r = bench.roofline({"refresh": (0.67, 1, 1.64e9, 0.0, 1)}, {})
    assert r["peak"] == 6800.0 and r["kernel"] == "refresh"


def test_roofline_of_the_fp64_small_solve():
    # the fused factor, inverse and product: tau^3 flops per slot, 600 slots
    fl = 600 * 256.0 ** 3
    r = bench.roofline({"potri": (12.8, 2, 1e8, fl, 2), "iterate": (0.585, 24, 1.6e8, 1e8, 1200)},
                       {"hbm_gbs": 6809.6})
    assert r["kernel"] == "potri" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - fl / 12.8e-3 / 1e12) < 1e-9
    assert r["peak"] == bench.FP64_PEAK_TFLOPS and abs(r["frac"] - r["achieved"] / 1.25) < 1e-12


def test_launch_count_of_a_mixed_step():
    # 1217 iterations in chunks of 600 with a refresh every 50: three chunks run, one
    # graph replay of four chunks; per chunk 6 phase-1 launches (M^+ in its two forms)
    # + 12 x (iterate + 3)
    assert bench.launches_per_step(1217, 600, 50) == 4 * (6 + 48) + 7
    # 2401 iterations: five chunks, two replays
    assert bench.launches_per_step(2401, 600, 50) == 8 * 54 + 7
    # factor and product as two launches
    assert bench.launches_per_step(100, 600, 50, fused=False) == 4 * 54 + 7
