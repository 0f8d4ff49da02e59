"""The allocation-free operator entry point (dwf_mdagm_noalloc), for callers that cannot
allocate device memory when they apply the operator.  On two calls in a row (the second reuses
the static scratch array the first one left behind) it must give the FP64 oracle's
A = Mpc^dag Mpc and what dwf_apply(MdagM) gives, within the operator tolerances of each
storage precision; once its kernels are loaded a call must not change the device's free
memory.  This file sorts last so that a run that stops at its first failure has already run
every other test."""
import numpy as np
import pytest

from oracle import dwf_oracle as o
from paper_1804_08593_gb300 import inputs
from tests.gpu_common import TOL, cuda, host, lib, rand_even, rel

pytestmark = pytest.mark.gpu

CASES = [
    # dims, Ls, M5, mf, b, c, eps: Moebius, Shamir, and D+ = b != 1 with c = 0
    ((4, 6, 2, 6), 6, 1.8, 0.05, 1.5, 0.5, 0.3),
    ((8, 8, 8, 8), 8, 1.8, 0.01, 1.0, 0.0, 0.3),
    ((4, 4, 4, 8), 4, 1.8, 0.1, 1.5, 0.0, 0.3),
]


@pytest.mark.parametrize("case", CASES, ids=["mobius", "shamir", "shamir_b1.5"])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_noalloc_matches_oracle_and_apply_on_two_calls(case, prec):
    import torch
    dwf = lib()
    dims, Ls, M5, mf, b, c, eps = case
    p = o.DWFParams(dims, Ls, M5, mf, b, c)
    rng = np.random.default_rng(41)
    Uh = inputs.gauge_links(dims, eps, rng)
    U = cuda(Uh)
    h = dwf.dwf_create(dims, Ls, M5, mf, b, c, U)
    for call in range(2):
        xh = rand_even(rng, dims, Ls)
        x = cuda(xh)
        ref = cuda(np.zeros(x.shape, complex))
        dwf.dwf_apply(h, "MdagM", x, ref, prec)
        out = cuda(np.full(x.shape, np.nan + 0j))
        dwf.dwf_mdagm_noalloc(dims, Ls, M5, mf, b, c, U, x, out, prec)
        torch.cuda.synchronize()
        got = host(out)
        assert rel(got, o.mdagm(Uh, xh, p)) <= TOL[prec], (call, prec, "oracle")
        assert rel(got, host(ref)) <= TOL[prec], (call, prec, "dwf_apply")


def test_noalloc_allocates_no_device_memory(monkeypatch):
    """After a first call has loaded its kernels (one fixed launch variant, so no new kernel is
    loaded later), a call leaves the device's free memory unchanged."""
    import torch
    dwf = lib()
    monkeypatch.setenv("DWF_STAGE_VARIANT", "0")
    dims, Ls = (8, 8, 4, 4), 8
    rng = np.random.default_rng(43)
    U = cuda(inputs.gauge_links(dims, 0.3, rng))
    x = cuda(rand_even(rng, dims, Ls))
    out = cuda(np.zeros(host(x).shape, complex))
    dwf.dwf_mdagm_noalloc(dims, Ls, 1.8, 0.05, 1.5, 0.5, U, x, out, "f32")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        dwf.dwf_mdagm_noalloc(dims, Ls, 1.8, 0.05, 1.5, 0.5, U, x, out, "f32")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_noalloc_rejects_oversized_lattice():
    dwf = lib()
    dims, Ls = (16, 16, 16, 16), 16
    U = cuda(inputs.unit_links(dims))
    x = cuda(np.zeros((Ls, 16 ** 4 // 2, 4, 3), complex))
    out = cuda(np.zeros_like(host(x)))
    with pytest.raises(dwf.DWFError) as e:
        dwf.dwf_mdagm_noalloc(dims, Ls, 1.8, 0.1, 1.0, 0.0, U, x, out, "f64")
    assert "too large" in str(e.value)
