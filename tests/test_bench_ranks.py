"""Host logic of bench.py's multi-rank path, on CPU with gloo (world size 2): every rank solves
its own replica; the reported time is the maximum over ranks; the reference arm runs on rank 0
only and the other ranks exit without work."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    got_ws, got_rank, _ = bench.dist_init()
    t = bench.max_over_ranks(1.5 + rank, got_ws)
    bench.barrier(got_ws)
    dist.destroy_process_group()
    q.put((got_rank, got_ws, t))


def test_max_over_ranks_gloo_world_size_2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 2.5), (1, 2, 2.5)]


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "cpu_model", lambda *a, **k: called.append(1))
    import oracle.dwf_oracle as o
    monkeypatch.setattr(o, "mdagm", lambda *a, **k: called.append(1))
    bench.run_reference(bench.argparse.Namespace(gpus=2, steps=1, warmup=0, local_op="exact",
                                                 l=6))
    assert not called and capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_0(monkeypatch, capsys):
    """Rank 0 times the oracle's A on the sample lattice (stubbed here by a fixed cost) and
    prints one JSON line with the reference fields."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    import oracle.dwf_oracle as o
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr(o, "mdagm", lambda *a, **k: None)
    bench.run_reference(bench.argparse.Namespace(gpus=1, steps=2, warmup=1, local_op="exact",
                                                 l=6))
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["higher_is_better"] is False
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] >= 0


def test_single_rank_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
