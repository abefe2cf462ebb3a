"""bench.py's measured DRAM traffic: an ncu capture is reported only for the launch form it was
taken of and only while the kernel sources hash to the value stored with it; the stored entries
are well formed and point at a committed profile summary."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_capture_reported_only_for_its_form_and_sources(monkeypatch):
    form = ("five_spot_4096", "staged_rows", 120)
    entry = {"bytes": 1234, "sources": "abc", "profile": "profiles/x.md"}
    monkeypatch.setattr(bench, "NCU_TRAFFIC_PER_LAUNCH", {form: entry})
    assert bench.captured_traffic(form, "abc") == (1234, "profiles/x.md")
    assert bench.captured_traffic(form, "abd") == (None, None)          # sources changed
    assert bench.captured_traffic(("five_spot_4096", "direct", 120), "abc") == (None, None)


def test_stored_captures_are_well_formed():
    for form, cap in bench.NCU_TRAFFIC_PER_LAUNCH.items():
        workload, kind, width = form
        assert workload in bench.WORKLOADS
        assert kind in set(bench.FUSED_FORM_NAMES.values()) | {"single"}
        assert isinstance(width, int)
        assert cap["bytes"] > 0 and len(cap["sources"]) == 16
        assert os.path.exists(os.path.join(ROOT, cap["profile"]))
        # the summary quotes the hash it was taken with
        assert cap["sources"] in open(os.path.join(ROOT, cap["profile"])).read()


def test_source_hash_covers_the_two_sweep_kernel_files():
    h = bench.kernel_source_hash("two_sweep")
    assert len(h) == 16 and int(h, 16) >= 0
    assert "sweep_rows.cu" in bench.KERNEL_SOURCES["two_sweep"]
