"""Builds libdwf.so (the CUDA kernels and the C ABI) in-tree for sm_103a with nvcc.

Each translation unit compiles in parallel; objects are rebuilt only when a source or header
is newer.  No torch headers are involved: the library depends on the CUDA runtime only.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "lib", "libdwf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
STAGE_PRECS = (0, 1, 2, 3)          # FP64, FP32, FP16, BF16
STAGE_LS = (4, 6, 8, 10, 12, 16)    # fifth-dimension extents with compiled stage kernels
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(h) for h in hs)


def build(verbose: bool = False, jobs: int | None = None, extra: list | None = None) -> str:
    """Compiles every csrc/*.cu and links lib/libdwf.so; returns the library path."""
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    # stage_ls.cu is compiled once per (storage precision, Ls, dag) and local_p.cu once per
    # storage precision: their kernel variants dominate the build, and the split lets them
    # compile in parallel
    units = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        if os.path.basename(src) == "local_p.cu":
            for p in STAGE_PRECS:
                units.append((src, [f"-DDWF_LOCAL_P={p}"], f"local_p{p}.o"))
        elif os.path.basename(src) == "stage_ls.cu":
            for p in STAGE_PRECS:
                for ls in STAGE_LS:
                    for dag in (0, 1):
                        units.append((src, [f"-DDWF_STAGE_P={p}", f"-DDWF_STAGE_LS={ls}",
                                            f"-DDWF_STAGE_DAG={dag}"],
                                      f"stage_p{p}_ls{ls}_d{dag}.o"))
        else:
            units.append((src, [], os.path.basename(src)[:-3] + ".o"))
    # the longest units first
    units.sort(key=lambda u: (not u[1], u[2]))
    hdr = _headers_mtime()
    cc = nvcc()
    extra = list(extra or [])

    def one(unit) -> str:
        src, defs, name = unit
        obj = os.path.join(BUILD, name)
        if os.path.exists(obj) and os.path.getmtime(obj) > max(os.path.getmtime(src), hdr):
            return obj
        cmd = [cc, *ARCH, *FLAGS, *defs, *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, flush=True)
        return obj

    jobs = jobs or min(len(units), max(2, os.cpu_count() or 2))
    with ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(one, units))
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [cc, *ARCH, "-shared", "-o", LIB, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv))
