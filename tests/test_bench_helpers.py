"""Host logic of the benchmark's measurement records (no GPU): the clock summary that decides
whether a run is rejected, and the roofline record's use of the committed ncu figures."""
import json
import os

import bench


def test_clock_summary_median_max_and_reasons():
    lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n",
        "0, 2055, 2070, 950.0, 0x4, Not Active, Not Active, Not Active, Active\n",
        "0, 1980, 2070, 1200.3, 0x8, Active, Not Active, Not Active, Not Active\n",
        "garbage line\n",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
    ]
    got = bench.ClockSampler.summarize(lines)
    assert got["samples"] == 3
    assert got["sm_mhz"] == 2055.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler.summarize(["no samples\n"]) is None


def test_roofline_scales_traffic_and_reports_issue_slots_only_for_the_captured_source():
    units = 74898195
    prof = {"reduce_fibers": (5, 94.0, 5 * units), "sggx_cluster": (45, 50.0, 100)}
    r = bench.roofline(prof, None, [1], 5)
    assert r["kernel"] == "reduce_fibers" and r["bound"] == "alu"
    ops = units * bench.ALU_OPS["reduce_fibers"]
    assert abs(r["achieved"] - ops / (18.8e-3) / 1e12) < 1e-9 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    ent = json.load(open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")))["reduce_fibers"]
    if ent["source_hash"] == bench._source_hash(ent["source"]):
        # the committed capture is of this source: traffic scaled by the units per launch
        want = ent["bytes_per_launch"] * units / ent["units_per_launch"]
        assert abs(r["traffic"] - want) < 1e-6 * want
        assert r["issue_slots"]["issue_active"] == ent["issue_active"]
    # a changed source drops both (the counters would describe another kernel)
    saved = bench._source_hash
    try:
        bench._source_hash = lambda name: "0" * 16
        r2 = bench.roofline(prof, None, [1], 5)
        assert r2["traffic"] is None and r2["issue_slots"] is None
    finally:
        bench._source_hash = saved


def test_roofline_hbm_stage_uses_the_byte_model():
    prof = {"sort_scatter": (3, 1.5, 3 * 1000000)}
    r = bench.roofline(prof, None, [1], 1)
    assert r["bound"] == "hbm"
    assert abs(r["achieved"] - 1000000 * bench.HBM_BYTES["sort_scatter"] / (0.5e-3) / 1e9) < 1e-6
