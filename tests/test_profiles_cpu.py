"""The committed profile summaries stay readable by bench.py: the per
cell-update counters line parses, names a 16-hex-digit fused-kernel
fingerprint and is found by bench.counters_from_profile for that fingerprint
only; every summary gives the command that made it."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PROFILES = os.path.join(ROOT, "profiles")


def _counter_rows():
    rows = []
    for line in open(os.path.join(PROFILES, "k_fused_c4_counters.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append(dict(x.split("=", 1) for x in line.split() if "=" in x))
    return rows


def test_counters_line_parses_and_is_found_by_fingerprint():
    rows = _counter_rows()
    assert rows, "no machine-readable counters line"
    for kv in rows:
        assert re.fullmatch(r"[0-9a-f]{16}", kv["build"])
        assert 288.0 <= float(kv["dram_bytes_per_cell_step"]) < 1000.0
        assert 0.0 < float(kv["warp_inst_per_cell_step"]) < 1000.0
        found = bench.counters_from_profile(kv["workload"], kv["build"])
        assert found == kv
    assert bench.counters_from_profile("c4", "0" * 16) == {}


def test_every_summary_gives_its_command():
    names = [f for f in os.listdir(PROFILES) if f.endswith((".md", ".txt"))]
    assert names
    for f in names:
        text = open(os.path.join(PROFILES, f)).read()
        assert "ncu " in text and "--clock-control none" in text, f
        assert "python bench.py" in text, f
        assert "_work" not in text, f
