"""Host logic of the profile summaries (no GPU): the ncu launch-list summary and the gate that
lets bench.py report recorded DRAM traffic only for the kernel source it was captured on."""
import glob
import os
import re

from paper_1804_08593_gb300 import profiling

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CSV_HEAD = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
            '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
            '"Metric Value"\n')


def _row(i, name, unit, value):
    return (f'"{i}","1","python3","h","{name}","1","7","(32, 6, 1)","(304, 1, 1)","0","10.3",'
            f'"Command line profiler metrics","gpu__time_duration.sum","{unit}","{value}"\n')


def test_launch_summary_counts_and_shares(tmp_path, capsys):
    p = tmp_path / "launches.csv"
    p.write_text("==PROF== Connected to process 1\n" + CSV_HEAD +
                 _row(0, "void dwf::stage_kernel<1, 12>(dwf::StageArgs)", "usecond", "300") +
                 _row(1, "void dwf::stage_kernel<1, 12>(dwf::StageArgs)", "nsecond", "300,000") +
                 _row(2, "void dwf::vec_kernel<1, 12>(dwf::VecArgs)", "usecond", "200") +
                 _row(3, "void dwf::cast_kernel<1, 2>(dwf::CastArgs)", "msecond", "0.2"))
    profiling.launches(str(p))
    out = capsys.readouterr().out
    lines = [ln for ln in out.splitlines() if ln.startswith("| `")]
    assert lines[0] == "| `dwf::stage_kernel<1, 12>` | 2 | 0.60 | 60.0% |"
    assert sorted(lines[1:]) == ["| `dwf::cast_kernel<1, 2>` | 1 | 0.20 | 20.0% |",
                                 "| `dwf::vec_kernel<1, 12>` | 1 | 0.20 | 20.0% |"]
    assert "4 launches, 1.0 ms" in out


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
