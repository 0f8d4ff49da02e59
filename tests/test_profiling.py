"""Host logic of the profile summaries (no GPU): the gate that lets bench.py report recorded
DRAM traffic only for the kernel source it was captured on."""
import glob
import os
import re

import bench as profiling

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

def test_traffic_reported_only_for_the_captured_source(tmp_path):
    sha = profiling.stage_sources_sha()
    assert re.fullmatch(r"[0-9a-f]{16}", sha)
    d = tmp_path / "profiles"
    d.mkdir()
    (d / "a.md").write_text(f"text\ntraffic: hop_f32_full_m5 123456 {sha}\n")
    (d / "b.md").write_text("traffic: hop_f16_halo 999 0123456789abcdef\n")
    assert profiling.recorded_traffic("hop_f32_full_m5", str(d)) == 123456
    assert profiling.recorded_traffic("hop_f16_halo", str(d)) is None     # other source
    assert profiling.recorded_traffic("hop_f32_full", str(d)) is None     # not recorded


def test_committed_traffic_lines_are_well_formed():
    pat = re.compile(r"^traffic:\s+(\S+)\s+(\d+)\s+([0-9a-f]{16})\s*$")
    n = 0
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(path):
            if line.startswith("traffic:"):
                assert pat.match(line.strip()), (path, line)
                n += 1
    assert n >= 1
