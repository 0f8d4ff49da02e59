#!/usr/bin/env python
"""Benchmark: time to solution at relative residual 1e-10 of mixed-precision MSPCG on the
Moebius 24^3x48 x Ls=12 workload (M5 = 1.8, mf = 0.005, b = 1.5, c = 0.5, links eps = 0.35,
seed 3; 512 blocks of 6^4, exact diagonal blocks P_s A P_s, l = 6 local CG iterations per
block in FP16 storage, FP32 outer CG, FP64 reliable updates), with the dominant kernel's
achieved HBM bandwidth against the measured roofline.

One step = one full solve A x = phi from x = 0 to ||phi - A x|| <= 1e-10 ||phi|| (true FP64
residual), inputs resident in HBM (every field is larger than the 129 MB L2, so no flush is
needed between steps).  The headline steps run without instrumentation; one more solve with
per-launch CUDA events gives the per-kernel figures and the roofline.  Also reported: the
end-to-end time through the C ABI with host buffers (links and source copied in, solution
copied out, every step), plain FP64 and mixed CG on the same GPU, the solution error against
a reference solve to 1e-14 and kappa(A) from the FP64 CG's Lanczos coefficients, the Shamir
16^4 x 16 workload with 8^4 blocks, the batched 64-problem workload, measured FP64/FP32 FMA
peaks, and the FP64 oracle timed on the host cores on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: replicas only (every rank solves its own instance; no collective in the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "mobius_24x24x24x48_ls12"
WORKLOAD_C2 = "shamir_16x16x16x16_ls16"
TOL = 1e-10
METRIC = "Time-to-solution @ rel resid 1e-10 (MSPCG mixed vs plain CG); Dslash HBM GB/s"
# FP64 CG iterations to 1e-10 on the 24^3x48 workload, measured with this library on a GB300
# (the oracle runs the same arithmetic, so it needs the same count); the reference arm, which
# cannot run the solve on the host in reasonable time, extrapolates with it.
CG_ITERS_MEASURED = 863
L_DEFAULT = 6    # local CG iterations per block (the paper's sloppy local solves, Sec. 4.1)


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--local-op", default="exact", choices=["exact", "drop"])
    ap.add_argument("--inner", default="f16", choices=["f16", "bf16", "f32"])
    ap.add_argument("--l", type=int, default=L_DEFAULT, help="local CG iterations per block")
    ap.add_argument("--quick", action="store_true",
                    help="headline, profiled pass and e2e only (no comparison runs)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--case", default="solve", choices=["solve", "apply", "precondition"],
                    help="apply: K applications of Mpc^dag Mpc; precondition: K MSPCG solves "
                         "with a small maxit (profiler captures)")
    ap.add_argument("--prec", default="f16", help="precision of --case apply")
    ap.add_argument("--dims", default=None,
                    help="X,Y,Z,T: a smaller lattice with the workload's other parameters, for "
                         "profiler captures (the JSON line then names that lattice)")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
STAGE_SOURCES = ("stage.cuh", "dwf_device.cuh", "tc_m5.cuh", "local_kernel.cuh", "sync.cuh")


def stage_sources_sha() -> str:
    """First 16 hex digits of the SHA-256 of the operator-kernel sources (stages, local solves)."""
    import hashlib
    h = hashlib.sha256()
    for name in STAGE_SOURCES:
        with open(os.path.join(ROOT, "paper_1804_08593_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_class: str, profiles_dir: str):
    """DRAM bytes per launch recorded for a kernel class in profiles/*.md, or None when none is
    recorded or the stage sources changed since the capture."""
    import glob
    import re
    sha = stage_sources_sha()
    pat = re.compile(r"^traffic:\s+(\S+)\s+(\d+)\s+([0-9a-f]+)\s*$")
    for path in sorted(glob.glob(os.path.join(profiles_dir, "*.md"))):
        with open(path) as f:
            for line in f:
                m = pat.match(line.strip().strip("`"))
                if m and m.group(1) == kernel_class and m.group(3) == sha:
                    return int(m.group(2))
    return None


def lanczos_kappa(res_hist, curv_hist):
    """Condition number of A from an uninterrupted CG run from x = 0 (the Lanczos connection):
    res_hist[k] = ||r_{k+1}|| / ||phi||, curv_hist[k] = <p_k, A p_k> / ||phi||^2.  With
    rho_k = ||r_k||^2 / ||phi||^2 (rho_0 = 1), alpha_k = rho_k / curv_k and
    beta_k = rho_{k+1} / rho_k, the Lanczos tridiagonal T has
      T[k, k] = 1/alpha_k + beta_{k-1}/alpha_{k-1},  T[k, k+1] = sqrt(beta_k) / alpha_k,
    and its extreme eigenvalues approximate those of A.  Returns (kappa, lambda_min,
    lambda_max)."""
    import numpy as np
    n = min(len(res_hist), len(curv_hist))
    rho = np.concatenate([[1.0], np.asarray(res_hist[:n], float) ** 2])
    curv = np.asarray(curv_hist[:n], float)
    alpha = rho[:n] / curv
    beta = rho[1:n + 1] / rho[:n]
    diag = 1.0 / alpha
    diag[1:] += beta[:n - 1] / alpha[:n - 1]
    off = np.sqrt(beta[:n - 1]) / alpha[:n - 1]
    T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    ev = np.linalg.eigvalsh(T)
    return float(ev[-1] / ev[0]), float(ev[0]), float(ev[-1])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        sm_sorted = sorted(sm)
        return {"sm_mhz": sm_sorted[len(sm) // 2] if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload.
# ------------------------------------------------------------------------------------------
SAMPLE_DIMS = (6, 6, 6, 12)   # 1/256 of the 24^3x48 volume, same Ls and parameters


def _oracle_apply_time(threads: int | None, reps: int) -> dict:
    """Times the oracle's A = Mpc^dag Mpc on the sample lattice in a fresh interpreter (so the
    thread limit of the numerical libraries takes effect); returns wall and CPU seconds per
    application."""
    code = f"""
import json, os, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
from oracle import dwf_oracle as o
from paper_1804_08593_gb300 import inputs
cfg = inputs.CONFIGS[{WORKLOAD!r}]
dims = {SAMPLE_DIMS!r}
rng = np.random.default_rng(cfg["seed"])
U = inputs.gauge_links(dims, cfg["eps"], rng)
phi = inputs.even_source(dims, cfg["Ls"], rng)
p = o.DWFParams(dims, cfg["Ls"], cfg["M5"], cfg["mf"], cfg["b"], cfg["c"])
o.mdagm(U, phi, p)
w0, c0 = time.perf_counter(), time.process_time()
for _ in range({reps}):
    o.mdagm(U, phi, p)
w1, c1 = time.perf_counter(), time.process_time()
print(json.dumps(dict(wall=(w1 - w0) / {reps}, cpu=(c1 - c0) / {reps})))
"""
    env = dict(os.environ)
    if threads:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = str(threads)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       check=True)
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_baseline(iters: int, reps: int = 3) -> dict:
    """The oracle's plain FP64 CG time to solution on the full workload, extrapolated from its
    A application on the sample lattice: (iters + 1) applications at 256x the sample's time
    (the oracle's operator is linear in the volume).  Timed with the numerical libraries free to
    use every core and limited to one thread; `cores` is the CPU time over wall time of the
    faster run (the threads it actually kept busy)."""
    import numpy as np
    vol = float(np.prod([24, 24, 24, 48])) / float(np.prod(SAMPLE_DIMS))
    all_c = _oracle_apply_time(None, reps)
    one = _oracle_apply_time(1, reps)
    best = all_c if all_c["wall"] <= one["wall"] else one
    cores = max(1, round(best["cpu"] / best["wall"]))
    per_apply = best["wall"] * vol
    return {"value": per_apply * (iters + 1), "unit": "s", "cores": cores, "kind": "oracle",
            "sample": (f"oracle A = Mpc^dag Mpc on {'x'.join(map(str, SAMPLE_DIMS))} x Ls=12 "
                       f"(1/{vol:.0f} of the volume, same parameters): {all_c['wall']:.3f} s "
                       f"per application with all threads allowed, {one['wall']:.3f} s with one "
                       f"(nproc {os.cpu_count()}, {cpu_model()}); x{vol:.0f} volume x "
                       f"{iters + 1} applications = plain FP64 CG to 1e-10 (extrapolated)"),
            "seconds_per_application_full_volume": per_apply,
            "threads_all": {"wall_s": all_c["wall"], "cpu_s": all_c["cpu"]},
            "threads_1": {"wall_s": one["wall"], "cpu_s": one["cpu"]}}


# ------------------------------------------------------------------------------------------
def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, ws: int) -> float:
    """Largest per-rank value over all ranks: every rank solves its own replica, so the job's
    time is the slowest rank's (NCCL reduces on the GPU, gloo on the host)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(a):
    """The oracle as the reference arm: every step times one A application of the FP64 oracle
    on the sample lattice; the value is the extrapolated plain-CG time to solution."""
    ws, rank, local = dist_init()
    if rank != 0:
        return
    import numpy as np

    from oracle import dwf_oracle as o
    from paper_1804_08593_gb300 import inputs
    t_run = time.time()
    cfg = inputs.CONFIGS[WORKLOAD]
    rng = np.random.default_rng(cfg["seed"])
    U = inputs.gauge_links(SAMPLE_DIMS, cfg["eps"], rng)
    phi = inputs.even_source(SAMPLE_DIMS, cfg["Ls"], rng)
    p = o.DWFParams(SAMPLE_DIMS, cfg["Ls"], cfg["M5"], cfg["mf"], cfg["b"], cfg["c"])
    vol = float(np.prod(cfg["dims"])) / float(np.prod(SAMPLE_DIMS))
    walls, cpus = [], []
    for i in range(a.warmup + a.steps):
        w0, c0 = time.perf_counter(), time.process_time()
        o.mdagm(U, phi, p)
        w1, c1 = time.perf_counter(), time.process_time()
        if i >= a.warmup:
            walls.append(w1 - w0)
            cpus.append(c1 - c0)
    wall = sorted(walls)[len(walls) // 2]
    cores = max(1, round(sum(cpus) / sum(walls)))
    value = wall * vol * (CG_ITERS_MEASURED + 1)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "solver": "plain CG (oracle)", "extrapolated": True},
        "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": (f"one oracle A = Mpc^dag Mpc per step on "
                                    f"{'x'.join(map(str, SAMPLE_DIMS))} x Ls=12 ({wall:.3f} s, "
                                    f"nproc {os.cpu_count()}, {cpu_model()}), x{vol:.0f} "
                                    f"volume x {CG_ITERS_MEASURED + 1} applications = plain "
                                    f"FP64 CG to 1e-10")},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.time() - t_run,
    }
    print(json.dumps(line), flush=True)


def load_workload(a):
    """The benchmark workload's parameters and fields (links, source); --dims swaps in another
    lattice drawn the same way (same seed and link spread)."""
    import numpy as np

    from paper_1804_08593_gb300 import inputs
    if not a.dims:
        return dict(inputs.CONFIGS[WORKLOAD]), inputs.workload(WORKLOAD)
    cfg = dict(inputs.CONFIGS[WORKLOAD])
    cfg["dims"] = tuple(int(v) for v in a.dims.split(","))
    rng = np.random.default_rng(cfg["seed"])
    w = dict(cfg)
    w["links"] = inputs.gauge_links(cfg["dims"], cfg["eps"], rng)
    w["phi"] = inputs.even_source(cfg["dims"], cfg["Ls"], rng)
    return cfg, w


def _sol_err(x, xref) -> float:
    import torch
    return float(torch.linalg.vector_norm(x - xref) / torch.linalg.vector_norm(xref))


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0


def _cg_study(dwf, h, phi_d, maxit=200000):
    """Plain FP64 CG to 1e-10 (time, iterations, kappa from its Lanczos coefficients), FP32 CG
    with FP64 reliable updates to 1e-10, and a reference solution to 1e-14 (FP32 CG with FP64
    reliable updates; its FP64 true residual is reported)."""
    import torch
    out = {}
    x64 = torch.zeros_like(phi_d)
    st, t = _timed(lambda: dwf.dwf_cg(h, phi_d, x64, TOL, maxit, "f64", history=maxit,
                                      curvature=True))
    kappa, lmin, lmax = lanczos_kappa(st["history"], st["curvature_history"])
    out["f64"] = {"seconds": t, "iterations": st["iterations"],
                  "true_residual": st["true_residual"]}
    out["kappa"] = {"value": kappa, "lambda_min": lmin, "lambda_max": lmax,
                    "from": f"Lanczos tridiagonal of the FP64 CG ({st['iterations']} steps)"}
    x32 = torch.zeros_like(phi_d)
    st, t = _timed(lambda: dwf.dwf_cg(h, phi_d, x32, TOL, maxit, "f32"))
    out["f32"] = {"seconds": t, "iterations": st["iterations"],
                  "reliable_updates": st["reliable_updates"], "true_residual": st["true_residual"]}
    xref = torch.zeros_like(phi_d)
    st = dwf.dwf_cg(h, phi_d, xref, 1e-14, maxit, "f32", raise_on_fail=False)
    out["reference_solution"] = {"solver": "f32 CG + f64 reliable updates", "tol": 1e-14,
                                 "true_residual": st["true_residual"]}
    out["f64"]["solution_error"] = _sol_err(x64, xref)
    out["f32"]["solution_error"] = _sol_err(x32, xref)
    return out, xref


def run_ours(a):
    import torch

    from paper_1804_08593_gb300 import build, dwf, inputs
    ws, rank, local = dist_init()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    dwf.load()
    cfg, w = load_workload(a)
    stream = torch.cuda.current_stream()
    links_d = torch.from_numpy(w["links"]).cuda()
    phi_d = torch.from_numpy(w["phi"]).cuda()
    h = dwf.dwf_create(cfg["dims"], cfg["Ls"], cfg["M5"], cfg["mf"], cfg["b"], cfg["c"],
                       links_d, stream)
    lop = dwf.LOCAL_EXACT if a.local_op == "exact" else dwf.LOCAL_DROP
    x = torch.zeros_like(phi_d)

    def solve(phi, xx, l=a.l):
        return dwf.dwf_mspcg(h, cfg["block"], l, a.inner, "f32", phi, xx, TOL, 20000,
                             local_op=lop)

    for _ in range(a.warmup):
        x.zero_()
        solve(phi_d, x)
    # headline: K solves, no per-launch instrumentation
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    ev0.record(stream)
    for _ in range(a.steps):
        x.zero_()
        stats.append(solve(phi_d, x))
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    t_step = max_over_ranks(ev0.elapsed_time(ev1) / 1e3 / a.steps, ws)

    # one more solve with CUDA events around every launch: per-kernel figures and roofline
    dwf.dwf_profile_enable(h, True)
    dwf.dwf_profile_read(h)
    xp = torch.zeros_like(phi_d)
    _, t_prof = _timed(lambda: solve(phi_d, xp))
    dwf.dwf_profile_enable(h, False)
    prof = dwf.dwf_profile_read(h)
    pk, pk_kind = peaks()
    prof.sort(key=lambda k: -k["ms"])
    top = prof[0]
    launches_per_solve = sum(k["launches"] for k in prof)
    achieved = top["bytes"] / top["launches"] / (top["ms"] / top["launches"] / 1e3) / 1e9
    hop = [k for k in prof if k["name"].startswith("hop_")]
    hop_ms = sum(k["ms"] for k in hop)
    hop32 = [k for k in hop if k["name"].startswith("hop_f32")]
    hop32_ms = sum(k["ms"] for k in hop32)
    total_ms = sum(k["ms"] for k in prof)

    # end to end through the C ABI with host buffers (links in, source in, solution out)
    e2e = None
    if not a.no_e2e:
        links_h = torch.from_numpy(w["links"]).pin_memory()
        phi_h = torch.from_numpy(w["phi"]).pin_memory()
        x_h = torch.zeros_like(phi_h).pin_memory()
        n_e2e = max(1, min(a.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            dwf.dwf_update_links(h, links_h)
            solve(phi_h, x_h)      # MSPCG starts from x = 0 and overwrites x
        torch.cuda.synchronize()
        e2e = {"value": (time.perf_counter() - t0) / n_e2e, "unit": "s", "steps": n_e2e,
               "h2d_bytes_per_step": int(links_h.numel() * 16 + phi_h.numel() * 16),
               "d2h_bytes_per_step": int(x_h.numel() * 16)}

    extra = {}
    if ws == 1 and not a.quick and not a.dims:
        cg, xref = _cg_study(dwf, h, phi_d)
        extra["plain_cg"] = cg
        extra["solution_error"] = {"mspcg": _sol_err(x, xref), "cg_f64": cg["f64"]["solution_error"],
                                   "cg_f32": cg["f32"]["solution_error"],
                                   "against": "reference solve to 1e-14"}
        extra["kappa"] = cg["kappa"]["value"]
        # the same solve with fewer local iterations (the paper's trade of g for local work)
        sweep = {}
        for lv in sorted({1, 2, a.l} - {a.l}):
            xs = torch.zeros_like(phi_d)
            st, t = _timed(lambda: solve(phi_d, xs, lv))
            sweep[f"l={lv}"] = {"seconds": t, "outer_iterations": st["iterations"],
                                "true_residual": st["true_residual"],
                                "solution_error": _sol_err(xs, xref)}
        extra["mspcg_other_l"] = sweep
        del xref
        # Shamir 16^4 x 16 (8^4 blocks, FP64 MSPCG with l = 6): g and solution errors
        w2 = inputs.workload(WORKLOAD_C2)
        h2 = dwf.dwf_create(w2["dims"], w2["Ls"], w2["M5"], w2["mf"], w2["b"], w2["c"],
                            torch.from_numpy(w2["links"]).cuda(), stream)
        phi2 = torch.from_numpy(w2["phi"]).cuda()
        cg2, xref2 = _cg_study(dwf, h2, phi2)
        c2 = {"workload": WORKLOAD_C2, "plain_cg": cg2, "kappa": cg2["kappa"]["value"]}
        for name, lo in (("mspcg_f64_drop", dwf.LOCAL_DROP), ("mspcg_f64_exact", dwf.LOCAL_EXACT)):
            xs = torch.zeros_like(phi2)
            st, t = _timed(lambda: dwf.dwf_mspcg(h2, w2["block"], w2["inner"], "f64", "f64",
                                                 phi2, xs, TOL, 20000, local_op=lo))
            c2[name] = {"seconds": t, "outer_iterations": st["iterations"], "l": w2["inner"],
                        "g": cg2["f64"]["iterations"] / max(1, st["iterations"]),
                        "true_residual": st["true_residual"],
                        "solution_error": _sol_err(xs, xref2)}
        extra["shamir_16x16x16x16_ls16"] = c2
        del h2, phi2, xref2
        # batched workload: 64 independent Moebius solves of uneven sizes in one call
        probs = []
        for pb in inputs.batch_problems(64, 4):
            U, ph = inputs.batch_problem_fields(pb)
            probs.append(dict(dims=pb["dims"], Ls=pb["Ls"], M5=pb["M5"], mf=pb["mf"], b=pb["b"],
                              c=pb["c"], links=torch.from_numpy(U).cuda(),
                              phi=torch.from_numpy(ph).cuda(),
                              x=torch.zeros(ph.shape, dtype=torch.complex128, device="cuda")))
        dwf.dwf_batch_solve(probs, TOL, 50000)          # first call: tuning, graph capture
        for pb in probs:
            pb["x"].zero_()
        bst, tb = _timed(lambda: dwf.dwf_batch_solve(probs, TOL, 50000))
        extra["batch"] = {"problems": len(probs), "seconds": tb, "solves_per_s": len(probs) / tb,
                          "iterations_total": int(sum(q["iterations"] for q in bst)),
                          "max_true_residual": max(q["true_residual"] for q in bst),
                          "precision": "f32 with f64 reliable updates"}
        del probs
        extra["measured_peaks"] = {"fp64_tflops": dwf.dwf_measure_peak("f64"),
                                   "fp32_tflops": dwf.dwf_measure_peak("f32"),
                                   "how": "independent FMA chains on every SM, CUDA events"}
        f64 = [k for k in prof if k["name"].startswith("hop_f64")]
        if f64 and sum(k["ms"] for k in f64) > 0:
            tf = sum(k["flops"] for k in f64) / (sum(k["ms"] for k in f64) / 1e3) / 1e12
            extra["fp64_stages"] = {"tflops": tf, "peak_tflops": extra["measured_peaks"]["fp64_tflops"],
                                    "frac": tf / extra["measured_peaks"]["fp64_tflops"],
                                    "flops": "1320 per site-slice"}

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu and not a.dims:
        iters = extra.get("plain_cg", {}).get("f64", {}).get("iterations", CG_ITERS_MEASURED)
        cpu = oracle_baseline(iters)

    s0 = stats[-1]
    bx = "x".join(str(v) for v in cfg["block"])
    line = {
        "metric": METRIC, "value": t_step, "unit": "s", "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": f"{a.inner}/f32/f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if not a.dims else WORKLOAD + " at " + a.dims,
                   "lattice": "x".join(str(v) for v in cfg["dims"]), "Ls": cfg["Ls"],
                   "solver": f"mspcg_{a.local_op}", "block": bx, "l": a.l,
                   "inner": a.inner, "middle": "f32", "outer": "f64", "tol": TOL,
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (764 MB source, no flush)"},
        "solve": {"outer_iterations": s0["iterations"], "inner_iterations": s0["inner_iterations"],
                  "reliable_updates": s0["reliable_updates"], "true_residual": s0["true_residual"]},
        "dslash": {"hbm_gbs": sum(k["bytes"] for k in hop) / (hop_ms / 1e3) / 1e9,
                   "gflops": sum(k["flops"] for k in hop) / (hop_ms / 1e3) / 1e9,
                   "share_of_step": hop_ms / total_ms,
                   "classes": "every outer-operator stage of the solve (FP32, and the FP64 "
                              "reliable updates, which the FP64 ALU bounds)",
                   "f32": {"hbm_gbs": sum(k["bytes"] for k in hop32) / (hop32_ms / 1e3) / 1e9,
                           "gflops": sum(k["flops"] for k in hop32) / (hop32_ms / 1e3) / 1e9,
                           "frac_of_hbm": (sum(k["bytes"] for k in hop32) / (hop32_ms / 1e3)
                                           / 1e9 / pk["hbm_gbs"])} if hop32_ms > 0 else None},
        "roofline": {"bound": "hbm", "kernel": top["name"], "achieved": achieved,
                     "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                     "peak_kind": pk_kind,
                     "traffic": recorded_traffic(top["name"], os.path.join(ROOT, "profiles")),
                     "launches": top["launches"], "avg_launch_ms": top["ms"] / top["launches"],
                     "share": top["ms"] / total_ms,
                     "measured": "CUDA events around every launch of one extra solve"},
        "kernels": [{"name": k["name"], "launches_per_solve": k["launches"],
                     "ms_per_solve": k["ms"],
                     "gbs": k["bytes"] / (k["ms"] / 1e3) / 1e9 if k["ms"] > 0 else None}
                    for k in prof],
        "profiled_solve_s": t_prof,
        "gpu_launches": launches_per_solve * a.steps,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    line.update(extra)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_apply(a):
    """K applications of Mpc^dag Mpc in one precision, or K short MSPCG solves (profiler
    captures of the operator and of the local-solve kernels)."""
    import torch

    from paper_1804_08593_gb300 import build, dwf, inputs
    torch.cuda.set_device(0)
    build.build()
    cfg, w = load_workload(a)
    h = dwf.dwf_create(cfg["dims"], cfg["Ls"], cfg["M5"], cfg["mf"], cfg["b"], cfg["c"],
                       torch.from_numpy(w["links"]).cuda())
    phi = torch.from_numpy(w["phi"]).cuda()
    out = torch.zeros_like(phi)
    for _ in range(a.warmup + a.steps):
        if a.case == "apply":
            dwf.dwf_apply(h, "MdagM", phi, out, a.prec)
        else:   # two outer iterations of the benchmark's MSPCG (three preconditioner steps)
            out.zero_()
            lop = dwf.LOCAL_EXACT if a.local_op == "exact" else dwf.LOCAL_DROP
            dwf.dwf_mspcg(h, cfg["block"], a.l, a.inner, "f32", phi, out, TOL, 2,
                          local_op=lop, raise_on_fail=False)
    torch.cuda.synchronize()
    print(json.dumps({"case": a.case, "prec": a.prec, "calls": a.warmup + a.steps}))


def main():
    a = args_parse()
    if a.case in ("apply", "precondition"):
        run_apply(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
