"""The benchmark's committed records stay tied to the sources they describe:
the headline kernel's DRAM-traffic record (profiles/traffic.json) carries
the hash of the sources it was captured from, and bench.py reports the
traffic only while that hash matches, so a kernel change without a new
capture shows up here instead of as a silent null."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_record_matches_the_kernel_sources():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    assert rec["kernel_hash"] == bench.kernel_hash(), "the headline kernel changed since its traffic was captured"
    assert rec["bytes_per_launch"] > 0
    assert "ncu" in rec["command"] and "--clock-control none" in rec["command"]


def test_roofline_denominators():
    # 152 SMs at 2070 MHz, 128 FP32 lanes: 2d + 2 = 6 operations per 2-D feature,
    # and the fast kernel's 2d + 1 = 5 packed ones
    assert abs(bench.alu_peak(152, 2070.0) - 152 * 2070e6 * 128 / 6) < 1.0
    assert abs(bench.kernel_pipe_peak(152, 2070.0) - 152 * 2070e6 * 128 / 5) < 1.0
    assert bench.alu_peak(152, 2070.0) < bench.kernel_pipe_peak(152, 2070.0)
