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
    # ncu traffic scaled to the iterations of one launch (400 here)
    assert abs(r["traffic"] - bench.PROFILED_TRAFFIC["iterate"](400)) < 1.0
    assert abs(r["traffic"] - 1802.8e6) < 1e3


def test_roofline_falls_back_without_measured_peaks():
    r = bench.roofline({"refresh": (0.67, 1, 1.64e9, 0.0, 1)}, {})
    assert r["peak"] == 6800.0 and r["kernel"] == "refresh"
