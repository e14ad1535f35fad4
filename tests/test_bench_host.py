"""Host-side helpers of bench.py that need no GPU: the instruction-issue
roofline of a count scan is the measured instructions per row scaled to the
launch, over 148 SMs x 4 schedulers x the SM clock, the shared-memory roofline
the measured wavefronts per row over 148 SMs x 1 wavefront a cycle; the algorithmic bytes of a
step count each predicate column of the batched scan once and each push-down's
reads and writes."""
import json
import os

import bench
import datagen as dg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_issue_roofline_scales_the_measured_instructions():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        entries = json.load(f)
    for kernel in ("bucket_count_kernel", "scan_count_kernel"):
        e = entries.get(kernel)
        r = bench.issue_roofline(kernel, 300_000_000, 5.0, 2000.0)
        if not e or "warp_instructions_per_row" not in e or e.get("source_hash") != bench.kernel_source_hash(kernel):
            assert r is None          # the capture no longer describes the kernel
            continue
        want = e["warp_instructions_per_row"] * 300_000_000 / 5e-3 / 1e9
        assert r["bound"] == "alu" and r["peak"] == 148 * 4 * 2.0
        assert abs(r["achieved"] - want) <= 0.05 + 1e-9 * want
        assert abs(r["frac"] - want / (148 * 4 * 2.0)) < 1e-4


def test_issue_roofline_needs_a_capture():
    assert bench.issue_roofline("bucket_count_kernel", 1000, 0.0, 2032.0) is None


def test_smem_roofline_scales_the_measured_wavefronts():
    """The shared-memory roofline: measured wavefronts per row scaled to the
    launch, over 148 SMs x 1 wavefront a cycle x the SM clock."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        e = json.load(f).get("bucket_count_kernel")
    r = bench.smem_roofline("bucket_count_kernel", 1_200_000_000, 50.0, 2000.0)
    if not e or "smem_wavefronts_per_row" not in e or e.get("source_hash") != bench.kernel_source_hash(
            "bucket_count_kernel"):
        assert r is None
        return
    want = e["smem_wavefronts_per_row"] * 1_200_000_000 / 50e-3 / 1e9
    assert r["bound"] == "smem" and r["peak"] == 148 * 2.0
    assert abs(r["achieved"] - want) <= 0.05 + 1e-9 * want
    assert abs(r["frac"] - want / (148 * 2.0)) < 1e-4
    assert bench.smem_roofline("bucket_count_kernel", 1000, 0.0, 2032.0) is None


def test_algorithmic_bytes_of_a_step():
    types = [s.type for s in dg.config5_specs()]
    trees = [dg.p_cmp(0, "<", 5), dg.p_and(dg.p_cmp(1, "=", 2), dg.p_cmp(3, "<", 1.0))]
    proj = [0, 1, 4]
    batch, pds = bench.algorithmic_bytes(types, 1000, trees, [10, 20], [0, 1], proj)
    assert batch == (4 + 4 + 4) * 1000                       # columns 0, 1, 3 once
    # probe 0 reads column 0; the selected rows' projected 1 and 4 (8 B); writes 3 x 4 B + 8 B row id
    assert pds[0] == 4 * 1000 + 10 * 8 + 10 * 20
    assert pds[1] == 8 * 1000 + 20 * 8 + 20 * 20             # projected 0 and 4 are not predicate columns
