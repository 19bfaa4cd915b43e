"""Host logic of the benchmark (no GPU): the clock summary taken during the
timed region, and the gate that reports a kernel's DRAM traffic only while
the committed ncu record matches the kernel sources and the box size."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

ROW = "0, {sm}, 2070, 812.50, 0x0000000000000000, {a}, {b}, {c}, {d}\n"


def test_clock_summary(tmp_path):
    p = tmp_path / "clocks.csv"
    na = "Not Active"
    p.write_text("index, clocks.sm [MHz], ...\n" + ROW.format(sm=2070, a=na, b=na, c=na, d=na)
                 + ROW.format(sm=1980, a=na, b=na, c=na, d="Active")
                 + ROW.format(sm=2070, a=na, b=na, c=na, d=na) + "garbage\n")
    s = bench.summarize_clocks(str(p))
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    p.write_text(ROW.format(sm=1400, a="Active", b=na, c="Active", d=na))
    assert bench.summarize_clocks(str(p))["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    p.write_text("no samples\n")
    assert bench.summarize_clocks(str(p)) is None


def test_traffic_is_reported_only_for_the_captured_sources_and_size(monkeypatch):
    rec = json.load(open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")))
    n = rec["cells"]
    # sources as they were when the record was taken
    monkeypatch.setattr(bench, "sources_sha256", lambda kind: rec["sources_sha256"][kind])
    for key in ("f32", "f16", "two_component"):
        assert bench.kernel_traffic(key, n) == rec[key]["bytes_per_launch_full"]
        assert bench.kernel_traffic(key, n // 4) is None  # another box size
    monkeypatch.setattr(bench, "sources_sha256", lambda kind: "0" * 64)  # the kernels changed
    for key in ("f32", "f16", "two_component"):
        assert bench.kernel_traffic(key, n) is None
