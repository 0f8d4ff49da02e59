"""The allocation-free operator entry point (dwf_mdagm_noalloc), for callers that cannot
allocate device memory when they apply the operator.  It must give what dwf_apply(MdagM)
gives, within the operator tolerances, on two calls in a row (the second call reuses the
static scratch array the first one left behind).  This file sorts last so that a run that
stops at its first failure has already run every other test."""
import numpy as np
import pytest

from paper_1804_08593_gb300 import inputs
from tests.gpu_common import TOL, cuda, host, lib, rand_even, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", [((4, 6, 2, 6), 6, 1.8, 0.05, 1.5, 0.5, 0.3),
                                  ((8, 8, 8, 8), 8, 1.8, 0.01, 1.0, 0.0, 0.3)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_matches_apply_on_two_calls(case, prec):
    import torch
    dwf = lib()
    dims, Ls, M5, mf, b, c, eps = case
    rng = np.random.default_rng(41)
    U = cuda(inputs.gauge_links(dims, eps, rng))
    h = dwf.dwf_create(dims, Ls, M5, mf, b, c, U)
    for call in range(2):
        x = cuda(rand_even(rng, dims, Ls))
        ref = cuda(np.zeros(x.shape, complex))
        dwf.dwf_apply(h, "MdagM", x, ref, prec)
        out = cuda(np.full(x.shape, np.nan + 0j))
        dwf.dwf_mdagm_noalloc(dims, Ls, M5, mf, b, c, U, x, out, prec)
        torch.cuda.synchronize()
        assert rel(host(out), host(ref)) <= TOL[prec], (call, prec)


def test_noalloc_rejects_oversized_lattice():
    dwf = lib()
    dims, Ls = (16, 16, 16, 16), 16
    U = cuda(inputs.unit_links(dims))
    x = cuda(np.zeros((Ls, 16 ** 4 // 2, 4, 3), complex))
    out = cuda(np.zeros_like(host(x)))
    with pytest.raises(dwf.DWFError) as e:
        dwf.dwf_mdagm_noalloc(dims, Ls, 1.8, 0.1, 1.0, 0.0, U, x, out, "f64")
    assert "too large" in str(e.value)
