"""The committed ncu traffic records agree with themselves and with the profile
summaries: read + write = total, every capture ran with --clock-control none,
and every capture named in a record is described in a summary under
profiles/ (host-side check; no GPU)."""
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROF = os.path.join(ROOT, "profiles")


def test_traffic_records_are_consistent_and_documented():
    with open(os.path.join(PROF, "traffic.json")) as fh:
        recs = json.load(fh)
    summaries = "".join(open(os.path.join(PROF, f)).read() for f in os.listdir(PROF) if f.endswith(".md"))
    assert recs
    for key, r in recs.items():
        assert r["dram_bytes_per_launch"] == r["dram_read_bytes_per_launch"] + r["dram_write_bytes_per_launch"], key
        assert "--clock-control none" in r["command"], key
        assert re.fullmatch(r"[0-9a-f]{16}", r["source_sha"]), key
        assert 0.0 <= r["l2_hit_rate"] <= 1.0, key
        out = re.search(r"-o (\S+)", r["command"]).group(1)
        assert out in summaries, (key, out)
        if "particles" in r:
            assert abs(r["dram_bytes_per_particle"] * r["particles"] - r["dram_bytes_per_launch"]) < r["particles"], key


def test_summaries_name_no_raw_reports():
    """Summaries are text; raw profiler reports are not committed."""
    for f in os.listdir(PROF):
        assert not f.endswith((".ncu-rep", ".nsys-rep", ".qdrep")), f
