"""Batched solver (dwf_batch_solve): many independent problems of different lattices, Ls,
masses and links in one call.  Every solution must reach the FP64 true residual (checked
with the oracle on the small problems) and match the single-problem FP64 CG solution."""
import numpy as np
import pytest

from oracle import dwf_oracle as o
from paper_1804_08593_gb300 import inputs
from tests.gpu_common import cuda, host, lib, rel

pytestmark = pytest.mark.gpu

SMALL = [  # dims, Ls, M5, mf, b, c, eps
    ((4, 4, 4, 4), 4, 1.8, 0.1, 1.5, 0.5, 0.3),
    ((4, 4, 4, 8), 8, 1.8, 0.05, 1.5, 0.5, 0.3),
    ((4, 6, 2, 6), 4, 1.8, 0.2, 1.0, 0.0, 0.3),      # Shamir, ragged tile
    ((6, 6, 6, 6), 8, 1.6, 0.03, 2.0, 1.0, 0.25),
    ((4, 4, 4, 4), 8, 1.8, 0.3, 1.0, 0.0, 0.2),
    ((8, 4, 4, 4), 12, 1.8, 0.02, 1.5, 0.5, 0.3),
]


def _problems(specs, seed):
    rng = np.random.default_rng(seed)
    out = []
    for dims, Ls, M5, mf, b, c, eps in specs:
        U = inputs.gauge_links(dims, eps, rng)
        phi = inputs.even_source(dims, Ls, rng)
        out.append(dict(dims=dims, Ls=Ls, M5=M5, mf=mf, b=b, c=c, U=U, phi=phi))
    return out


@pytest.mark.parametrize("form", ["tuned", "persistent", "stages"])
@pytest.mark.parametrize("host_buffers", [False, True])
def test_batch_matches_single_solves(host_buffers, form, monkeypatch):
    """Each form of a chunk of CG steps: one persistent launch per Ls group, one launch per
    stage, or whichever the tuner picks.  The second call of each form (host buffers after
    device buffers, same problems) reuses the form the first one picked."""
    if form != "tuned":
        monkeypatch.setenv("DWF_BATCH_FORM", form)
    dwf = lib()
    probs = _problems(SMALL, 51)
    batch = []
    for p in probs:
        if host_buffers:
            batch.append(dict(p, links=p["U"], phi=p["phi"], x=np.zeros_like(p["phi"])))
        else:
            batch.append(dict(p, links=cuda(p["U"]), phi=cuda(p["phi"]),
                              x=cuda(np.zeros_like(p["phi"]))))
    stats = dwf.dwf_batch_solve(batch, 1e-10, 20000)
    for p, b, st in zip(probs, batch, stats):
        x = b["x"] if host_buffers else host(b["x"])
        prm = o.DWFParams(p["dims"], p["Ls"], p["M5"], p["mf"], p["b"], p["c"])
        assert st["true_residual"] <= 1e-10
        assert o.true_residual(p["U"], x, p["phi"], prm) <= 1.5e-10
        h = dwf.dwf_create(p["dims"], p["Ls"], p["M5"], p["mf"], p["b"], p["c"], cuda(p["U"]))
        xs = cuda(np.zeros_like(p["phi"]))
        dwf.dwf_cg(h, cuda(p["phi"]), xs, 1e-12, 20000, "f64")
        assert rel(x, host(xs)) <= 1e-7


@pytest.mark.parametrize("form", ["tuned", "persistent"])
def test_batch_64_uneven_problems(form, monkeypatch):
    """The 64-problem Moebius workload (lattices 8^4, 8^3x16, 12^4, 16^3x32; Ls 8/12/16;
    mf in [0.005, 0.05]; eps in [0.2, 0.4]; seed 4): every problem reaches 1e-10 and a sample
    agrees with single-problem solves."""
    if form != "tuned":
        monkeypatch.setenv("DWF_BATCH_FORM", form)
    dwf = lib()
    specs = inputs.batch_problems(64, 4)
    batch = []
    for p in specs:
        U, phi = inputs.batch_problem_fields(p)
        batch.append(dict(dims=p["dims"], Ls=p["Ls"], M5=p["M5"], mf=p["mf"], b=p["b"], c=p["c"],
                          links=cuda(U), phi=cuda(phi), x=cuda(np.zeros_like(phi)), U=U, phi_h=phi))
    stats = dwf.dwf_batch_solve(batch, 1e-10, 50000)
    assert all(st["true_residual"] <= 1e-10 for st in stats)
    for k in (0, 17, 63):
        b = batch[k]
        h = dwf.dwf_create(b["dims"], b["Ls"], b["M5"], b["mf"], b["b"], b["c"], b["links"])
        r = cuda(np.zeros_like(b["phi_h"]))
        dwf.dwf_apply(h, "MdagM", b["x"], r, "f64")
        res = np.linalg.norm(host(r) - b["phi_h"]) / np.linalg.norm(b["phi_h"])
        assert res <= 1.5e-10
