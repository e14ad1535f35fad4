"""Host-side helpers of bench.py that need no GPU: the instruction-issue
roofline of the count scan is the measured instructions per row scaled to the
launch, over 148 SMs x 4 schedulers x the SM clock."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_issue_roofline_scales_the_measured_instructions():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        e = json.load(f)["scan_count_kernel"]
    r = bench.issue_roofline("scan_count_kernel", "count.cu", 300_000_000, 5.0, 2000.0)
    if e.get("source_hash") != bench.kernel_source_hash("count.cu"):
        assert r is None          # the capture no longer describes the kernel
        return
    want = e["warp_instructions_per_row"] * 300_000_000 / 5e-3 / 1e9
    assert r["bound"] == "alu" and r["peak"] == 148 * 4 * 2.0
    assert abs(r["achieved"] - want) <= 0.05 + 1e-9 * want
    assert abs(r["frac"] - want / (148 * 4 * 2.0)) < 1e-4


def test_issue_roofline_needs_a_capture():
    assert bench.issue_roofline("no_such_kernel", "count.cu", 1000, 1.0, 2032.0) is None
    assert bench.issue_roofline("scan_count_kernel", "count.cu", 1000, 0.0, 2032.0) is None
