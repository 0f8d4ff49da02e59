"""Helpers for the ncu summaries kept under profiles/ and for bench.py's roofline entry.

  python -m paper_1804_08593_gb300.profiling launches <launches.csv>  # per kernel: launches, time, share
  python -m paper_1804_08593_gb300.profiling report <file.ncu-rep>    # key counters per captured launch
  python -m paper_1804_08593_gb300.profiling sha                      # hash of the stage-kernel sources

The launch list comes from
  ncu --metrics gpu__time_duration.sum --clock-control none -c <N> --csv --log-file <csv> <cmd>
and the report from
  ncu --set full --clock-control none -k regex:<kernel> -s <n> -c <m> -o <file> <cmd>.
A summary that records DRAM traffic per launch carries a line
  traffic: <kernel class> <bytes per launch> <sha>
where <sha> is stage_sources_sha() at capture time; bench.py reports the traffic only while
the stage sources still hash to it.
"""
from __future__ import annotations

import collections
import csv
import glob
import hashlib
import io
import os
import re
import subprocess
import sys

COUNTERS = [
    "gpu__time_duration.sum", "dram__bytes_read.sum", "dram__bytes_write.sum",
    "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed",
    "sm__throughput.avg.pct_of_peak_sustained_elapsed", "sm__warps_active.avg.per_cycle_active",
    "launch__registers_per_thread", "launch__shared_mem_per_block_dynamic",
    "smsp__inst_executed.sum", "l1tex__t_sector_hit_rate.pct", "lts__t_sector_hit_rate.pct",
    "sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active",
    "smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio",
    "smsp__issue_active.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_fma.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_fp64.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active",
    "launch__grid_size",
]


def launches(path: str) -> None:
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hi]
    ki, mi, vi, ui = (hdr.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value",
                                             "Metric Unit"))
    agg = collections.defaultdict(lambda: [0, 0.0])
    scale = {"ns": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0,
             "nsecond": 1e-6}
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        ms = float(r[vi].replace(",", "")) * scale.get(r[ui], 1e-6)
        name = r[ki].split("(")[0].replace("void ", "")
        agg[name][0] += 1
        agg[name][1] += ms
    tot = sum(v[1] for v in agg.values())
    print("| kernel | launches | total ms | share |")
    print("|---|---:|---:|---:|")
    for k, v in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print(f"| `{k}` | {v[0]} | {v[1]:.2f} | {100 * v[1] / tot:.1f}% |")
    print(f"\n{sum(v[0] for v in agg.values())} launches, {tot:.1f} ms (serialised, cold-cache)")


def report(path: str) -> None:
    out = subprocess.run(["ncu", "-i", path, "--page", "raw", "--csv"], capture_output=True,
                         text=True, check=True).stdout
    rows = list(csv.reader(io.StringIO(out)))
    hdr, units = rows[0], rows[1]
    for r in rows[2:]:
        print(f"### `{r[hdr.index('Kernel Name')]}`\n")
        print("| counter | value |")
        print("|---|---|")
        for c in COUNTERS:
            if c in hdr:
                i = hdr.index(c)
                print(f"| {c} | {r[i]} {units[i]} |")
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
        dram = 0.0
        for c in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            if c in hdr:
                i = hdr.index(c)
                dram += float(r[i].replace(",", "")) * scale.get(units[i], 1)
        print(f"| DRAM bytes (read + write) | {dram:.0f} |")
        print()


HERE = os.path.dirname(os.path.abspath(__file__))
STAGE_SOURCES = ("stage.cuh", "dwf_device.cuh", "tc_m5.cuh")   # the kernel code itself


def stage_sources_sha() -> str:
    """First 16 hex digits of the SHA-256 of the stage-kernel sources."""
    h = hashlib.sha256()
    for name in STAGE_SOURCES:
        with open(os.path.join(HERE, "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_class: str, profiles_dir: str):
    """DRAM bytes per launch recorded for a kernel class in profiles/*.md, or None when none is
    recorded or the stage sources changed since the capture."""
    sha = stage_sources_sha()
    pat = re.compile(r"^traffic:\s+(\S+)\s+(\d+)\s+([0-9a-f]+)\s*$")
    for path in sorted(glob.glob(os.path.join(profiles_dir, "*.md"))):
        with open(path) as f:
            for line in f:
                m = pat.match(line.strip().strip("`"))
                if m and m.group(1) == kernel_class and m.group(3) == sha:
                    return int(m.group(2))
    return None


if __name__ == "__main__":
    if sys.argv[1] == "sha":
        print(stage_sources_sha())
    else:
        {"launches": launches, "report": report}[sys.argv[1]](sys.argv[2])
