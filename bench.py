#!/usr/bin/env python
"""Benchmark: time to solution at relative residual 1e-10 of mixed-precision MSPCG on the
Moebius 24^3x48 x Ls=12 workload (M5 = 1.8, mf = 0.005, b = 1.5, c = 0.5, links eps = 0.35,
seed 3; 512 blocks of 6^4, exact diagonal blocks P_s A P_s, l local iterations in FP16 storage
(l = 1 by default, the fastest on one GPU), FP32 outer CG, FP64 reliable updates), with the
operator stage's achieved HBM bandwidth against the measured roofline.

One step = one full solve A x = phi from x = 0 to ||phi - A x|| <= 1e-10 ||phi|| (true FP64
residual), inputs resident in HBM (every field is larger than the 129 MB L2, so no flush is
needed between steps).  Also reported: the end-to-end time through the C ABI with host
buffers (links and source copied in, solution copied out, every step), plain FP64 CG on the
same GPU (--with-cg), the per-kernel roofline from CUDA events recorded around every launch
in the timed region, and the FP64 oracle timed on the host cores on a bounded sample.

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
TOL = 1e-10
METRIC = "Time-to-solution @ rel resid 1e-10 (MSPCG mixed vs plain CG); Dslash HBM GB/s"
# Outer MSPCG iterations to 1e-10 on this workload (exact blocks, l = 1, FP16 inner), measured
# with this library on a GB300; used only to extrapolate the oracle's per-iteration time in the
# reference arm, which cannot run the solve itself.
OUTER_ITERS_MEASURED = 878


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--local-op", default="exact", choices=["exact", "drop"])
    ap.add_argument("--inner", default="f16", choices=["f16", "bf16", "f32"])
    ap.add_argument("--l", type=int, default=1,
                    help="local CG iterations per block (1 is fastest on one GB300: see DESIGN)")
    ap.add_argument("--no-cg", action="store_true",
                    help="skip the plain-CG comparison (FP64 CG and FP32 CG with FP64 updates)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched workload (64 uneven Moebius solves in one call)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the MSPCG runs with more local iterations (l = 2, 6)")
    ap.add_argument("--case", default="solve", choices=["solve", "apply"],
                    help="apply: only K applications of Mpc^dag Mpc (for profiler captures)")
    ap.add_argument("--prec", default="f16", help="precision of --case apply")
    ap.add_argument("--dims", default=None,
                    help="X,Y,Z,T: a smaller lattice with the workload's other parameters, for "
                         "profiler captures (the JSON line then names that lattice)")
    return ap.parse_args()


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
def oracle_sample(local_op: str, l: int, reps: int = 1):
    """Times the oracle's A application and block preconditioner on a 6^3x12 x Ls=12 lattice
    (1/256 of the workload's volume, same parameters, two 6^4 blocks) and scales them to the
    full volume; returns (seconds per outer iteration at full size, description, threads)."""
    import numpy as np

    from oracle import dwf_oracle as o
    from paper_1804_08593_gb300 import inputs
    cfg = inputs.CONFIGS[WORKLOAD]
    dims = (6, 6, 6, 12)
    rng = np.random.default_rng(cfg["seed"])
    U = inputs.gauge_links(dims, cfg["eps"], rng)
    phi = inputs.even_source(dims, cfg["Ls"], rng)
    p = o.DWFParams(dims, cfg["Ls"], cfg["M5"], cfg["mf"], cfg["b"], cfg["c"])
    block = cfg["block"]
    eb = o.even_block_ids(dims, block)
    nb_s = int(np.prod([dims[i] // block[i] for i in range(4)]))
    nb_f = int(np.prod([cfg["dims"][i] // block[i] for i in range(4)]))
    if local_op == "exact":
        apply_blk = o.exact_block_operator(U, p, block)
    else:
        Ub = o.block_links(U, dims, block)

        def apply_blk(v):
            return o.mdagm(Ub, v, p)
    t_a = t_p = 0.0
    for _ in range(reps):
        t0 = time.perf_counter()
        o.mdagm(U, phi, p)
        t1 = time.perf_counter()
        o.block_cg(apply_blk, phi, eb, nb_s, l)
        t2 = time.perf_counter()
        t_a += t1 - t0
        t_p += t2 - t1
    t_a /= reps
    t_p /= reps
    vol = float(np.prod(cfg["dims"])) / float(np.prod(dims))
    # the oracle's exact block operator applies A once per block, so its cost grows with the
    # number of blocks as well as with the volume
    scale_p = vol * (nb_f / nb_s if local_op == "exact" else 1.0)
    per_iter = t_a * vol + t_p * scale_p
    threads = os.cpu_count()
    desc = (f"oracle A application + one {local_op}-block preconditioner (l={l}) on "
            f"6x6x6x12 x Ls=12 ({t_a:.2f}s + {t_p:.2f}s), scaled x{vol:.0f} volume"
            f"{' x%d blocks' % (nb_f // nb_s) if local_op == 'exact' else ''} to one outer "
            f"iteration of the full workload")
    return per_iter, desc, threads


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
    ws, rank, local = dist_init()
    if rank != 0:
        return
    t_run = time.time()
    per_iter = None
    samples = []
    for i in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        per_iter, desc, threads = oracle_sample(a.local_op, a.l)
        if i >= a.warmup:
            samples.append(per_iter)
    value = sorted(samples)[len(samples) // 2] * OUTER_ITERS_MEASURED
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "solver": f"mspcg_{a.local_op}", "l": a.l,
                   "extrapolated": True},
        "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle",
                         "sample": desc + f" x {OUTER_ITERS_MEASURED} outer iterations"},
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


def run_ours(a):
    import numpy as np
    import torch

    from paper_1804_08593_gb300 import build, dwf, inputs, profiling
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

    def solve(phi, xx):
        return dwf.dwf_mspcg(h, cfg["block"], a.l, a.inner, "f32", phi, xx, TOL, 20000,
                             local_op=lop)

    for _ in range(a.warmup):
        x.zero_()
        solve(phi_d, x)
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    dwf.dwf_profile_enable(h, True)
    dwf.dwf_profile_read(h)
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
    dwf.dwf_profile_enable(h, False)
    prof = dwf.dwf_profile_read(h)
    ms = ev0.elapsed_time(ev1)
    t_step = ms / 1e3 / a.steps
    t_step = max_over_ranks(t_step, ws)

    # roofline of the dominant kernel class
    pk, pk_kind = peaks()
    prof.sort(key=lambda k: -k["ms"])
    top = prof[0]
    launches = sum(k["launches"] for k in prof)
    achieved = top["bytes"] / top["launches"] / (top["ms"] / top["launches"] / 1e3) / 1e9
    hop = [k for k in prof if k["name"].startswith("hop_")]
    hop_gbs = sum(k["bytes"] for k in hop) / (sum(k["ms"] for k in hop) / 1e3) / 1e9
    hop_gflops = sum(k["flops"] for k in hop) / (sum(k["ms"] for k in hop) / 1e3) / 1e9
    total_ms = sum(k["ms"] for k in prof)

    # end to end through the C ABI with host buffers (links in, source in, solution out)
    e2e = None
    if not a.no_e2e:
        links_h = torch.from_numpy(w["links"]).pin_memory()
        phi_h = torch.from_numpy(w["phi"]).pin_memory()
        x_h = torch.zeros_like(phi_h).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            dwf.dwf_update_links(h, links_h)
            solve(phi_h, x_h)      # MSPCG starts from x = 0 and overwrites x
        torch.cuda.synchronize()
        e2e_t = (time.perf_counter() - t0) / a.steps
        e2e = {"value": e2e_t, "unit": "s",
               "h2d_bytes_per_step": int(links_h.numel() * 16 + phi_h.numel() * 16),
               "d2h_bytes_per_step": int(x_h.numel() * 16)}

    plain_cg = {}
    if not a.no_cg:
        for prec in ("f64", "f32"):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = dwf.dwf_cg(h, phi_d, x, TOL, 100000, prec)
            torch.cuda.synchronize()
            plain_cg[prec] = {"seconds": time.perf_counter() - t0,
                              "iterations": st["iterations"],
                              "reliable_updates": st["reliable_updates"],
                              "true_residual": st["true_residual"]}

    # the same solve with more local iterations: the paper's trade of global iterations (g)
    # for local work, for comparison with the default
    sweep = {}
    if not a.no_sweep:
        for lv in (2, 6):
            xs = torch.zeros_like(phi_d)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = dwf.dwf_mspcg(h, cfg["block"], lv, a.inner, "f32", phi_d, xs, TOL, 20000,
                               local_op=lop)
            torch.cuda.synchronize()
            sweep[f"l={lv}"] = {"seconds": time.perf_counter() - t0,
                                "outer_iterations": st["iterations"],
                                "true_residual": st["true_residual"]}

    # batched workload: 64 independent Moebius solves of uneven sizes in one call
    batch = None
    if not a.no_batch:
        probs = []
        for p in inputs.batch_problems(64, 4):
            U, ph = inputs.batch_problem_fields(p)
            probs.append(dict(dims=p["dims"], Ls=p["Ls"], M5=p["M5"], mf=p["mf"], b=p["b"],
                              c=p["c"], links=torch.from_numpy(U).cuda(),
                              phi=torch.from_numpy(ph).cuda(),
                              x=torch.zeros(ph.shape, dtype=torch.complex128, device="cuda")))
        dwf.dwf_batch_solve(probs, TOL, 50000)          # first call: tuning, graph capture
        for p in probs:
            p["x"].zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bst = dwf.dwf_batch_solve(probs, TOL, 50000)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        batch = {"problems": len(probs), "seconds": tb, "solves_per_s": len(probs) / tb,
                 "iterations_total": int(sum(s["iterations"] for s in bst)),
                 "max_true_residual": max(s["true_residual"] for s in bst),
                 "precision": "f32 with f64 reliable updates"}

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu:
        per_iter, desc, threads = oracle_sample(a.local_op, a.l)
        iters = stats[-1]["iterations"]
        cpu = {"value": per_iter * iters, "unit": "s", "cores": threads, "kind": "oracle",
               "sample": desc + f" x {iters} outer iterations (extrapolated)"}

    s0 = stats[-1]
    line = {
        "metric": METRIC, "value": t_step, "unit": "s", "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": f"{a.inner}/f32/f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if not a.dims else WORKLOAD + " at " + a.dims,
                   "lattice": "x".join(str(v) for v in cfg["dims"]), "Ls": cfg["Ls"],
                   "solver": f"mspcg_{a.local_op}", "block": "6x6x6x6", "l": a.l,
                   "inner": a.inner, "middle": "f32", "outer": "f64", "tol": TOL,
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (764 MB source, no flush)"},
        "solve": {"outer_iterations": s0["iterations"], "inner_iterations": s0["inner_iterations"],
                  "reliable_updates": s0["reliable_updates"], "true_residual": s0["true_residual"]},
        "dslash": {"hbm_gbs": hop_gbs, "gflops": hop_gflops,
                   "share_of_step": sum(k["ms"] for k in hop) / total_ms},
        "roofline": {"bound": "hbm", "kernel": top["name"], "achieved": achieved,
                     "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                     "peak_kind": pk_kind,
                     "traffic": profiling.recorded_traffic(top["name"],
                                                           os.path.join(ROOT, "profiles")),
                     "launches": top["launches"] // a.steps,
                     "avg_launch_ms": top["ms"] / top["launches"],
                     "share": top["ms"] / total_ms},
        "kernels": [{"name": k["name"], "launches_per_step": k["launches"] // a.steps,
                     "ms_per_step": k["ms"] / a.steps,
                     "gbs": k["bytes"] / (k["ms"] / 1e3) / 1e9 if k["ms"] > 0 else None}
                    for k in prof],
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if plain_cg:
        line["plain_cg"] = plain_cg
    if batch:
        line["batch"] = batch
    if sweep:
        line["mspcg_more_local_iterations"] = sweep
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_apply(a):
    """K applications of Mpc^dag Mpc on the workload in one precision (profiler captures)."""
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
        dwf.dwf_apply(h, "MdagM", phi, out, a.prec)
    torch.cuda.synchronize()
    print(json.dumps({"case": "apply", "prec": a.prec, "applications": a.warmup + a.steps}))


def main():
    a = args_parse()
    if a.case == "apply":
        run_apply(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
