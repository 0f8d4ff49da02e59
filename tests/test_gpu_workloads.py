"""The named workloads at their full sizes, in the launch configurations the solvers and the
benchmark use, checked where the whole-lattice oracle would take too long:

* operator parity at sampled sites: Mpc and Mpc^dag of the workload's own source field on
  the GPU against the oracle evaluated site by site (oracle.mpc_at_sites), to the operator
  tolerances (FP64 1e-13, FP32 1e-6, FP16/BF16 5e-3 relative over the sample);
* Shamir 16^4 x 16: plain FP64 CG and FP64 MSPCG (2^4 blocks of 8^4 with the hopping across
  block faces dropped, 6 local iterations) both reach relative residual 1e-10, with the true
  residual recomputed by the oracle on the whole lattice, and agree with each other to the
  accuracy the conditioning allows."""
import numpy as np
import pytest

from oracle import dwf_oracle as o
from paper_1804_08593_gb300 import inputs
from tests.gpu_common import TOL, cuda, host, lib

pytestmark = pytest.mark.gpu

_cache = {}


def _workload(name):
    if name not in _cache:
        dwf = lib()
        w = inputs.workload(name)
        p = o.DWFParams(w["dims"], w["Ls"], w["M5"], w["mf"], w["b"], w["c"])
        h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(w["links"]))
        _cache[name] = (w, p, h)
    return _cache[name]


def _sample(n, k, seed):
    rng = np.random.default_rng(seed)
    return sorted(set([0, n - 1] + list(rng.choice(n, size=k, replace=False))))


@pytest.mark.parametrize("name", ["shamir_16x16x16x16_ls16", "mobius_24x24x24x48_ls12"])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_full_size_operator_at_sampled_sites(name, prec):
    dwf = lib()
    w, p, h = _workload(name)
    x = w["phi"]
    sites = _sample(x.shape[1], 40, 7)
    dx = cuda(x)
    out = cuda(np.zeros_like(x))
    for op, dag in (("Mpc", False), ("Mpc_dag", True)):
        dwf.dwf_apply(h, op, dx, out, prec)
        got = host(out)[:, sites]
        ref = o.mpc_at_sites(w["links"], x, p, sites, dag)
        err = float(np.linalg.norm((got - ref).reshape(-1)) / np.linalg.norm(ref.reshape(-1)))
        assert err <= TOL[prec], (name, op, prec, err)


def test_shamir_16_plain_cg_and_mspcg_fp64():
    dwf = lib()
    w, p, h = _workload("shamir_16x16x16x16_ls16")
    phi = cuda(w["phi"])
    x_cg = cuda(np.zeros_like(w["phi"]))
    st_cg = dwf.dwf_cg(h, phi, x_cg, 1e-10, 20000, "f64")
    x_ms = cuda(np.zeros_like(w["phi"]))
    st_ms = dwf.dwf_mspcg(h, w["block"], w["inner"], "f64", "f64", phi, x_ms, 1e-10, 20000,
                          local_op=dwf.LOCAL_DROP)
    assert st_cg["true_residual"] <= 1e-10 and st_ms["true_residual"] <= 1e-10
    a, b = host(x_cg), host(x_ms)
    for xx in (a, b):
        assert o.true_residual(w["links"], xx, w["phi"], p) <= 1.01e-10
    # ||x_cg - x_ms|| / ||x|| <= kappa * 2e-10; kappa of Mpc^dag Mpc here is O(1e4)
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(a)
