"""Stationary block iterations (dwf_ms_solve): the multisplitting iteration of Sec. 2.1
(Eq. 2; colours = 1, all blocks at once) and multiplicative Schwarz sweeps over the 2- and
16-colour checkerboards of blocks (Sec. 1.2).  With FP64 local solves every sweep must follow
the oracle's ms_solve (residual history to 1e-6 relative, solution to 1e-9 after the same
number of sweeps); with FP16 local solves the residual after the sweeps must be close to the
oracle's FP64 one."""
import numpy as np
import pytest

from oracle import dwf_oracle as o
from paper_1804_08593_gb300 import inputs
from tests.gpu_common import cuda, host, lib, rel

pytestmark = pytest.mark.gpu

CASES = {
    # name: dims, Ls, block, (b, c), mf, local iterations, colours, sweeps, seed
    "additive_mobius": ((4, 4, 4, 4), 4, (2, 2, 2, 2), (1.5, 0.5), 0.3, 3, 1, 4, 41),
    "sap2_mobius": ((4, 4, 4, 4), 4, (2, 2, 2, 2), (1.5, 0.5), 0.3, 3, 2, 3, 42),
    "col16_shamir": ((4, 4, 4, 4), 4, (2, 2, 2, 2), (1.0, 0.0), 0.3, 2, 16, 2, 43),
    "sap2_8x4_blocks": ((8, 4, 4, 4), 4, (4, 4, 2, 2), (1.5, 0.5), 0.2, 2, 2, 2, 44),
}
_cache = {}


def case(name):
    if name not in _cache:
        dims, Ls, blk, (b, c), mf, l, ncol, n, seed = CASES[name]
        rng = np.random.default_rng(seed)
        p = o.DWFParams(dims, Ls, 1.8, mf, b, c)
        U = inputs.gauge_links(dims, 0.3, rng)
        phi = inputs.even_source(dims, Ls, rng)
        xo, ko, hist = o.ms_solve(U, phi, p, blk, l, ncol, 0.0, n)
        _cache[name] = (p, U, phi, blk, l, ncol, n, xo, hist)
    return _cache[name]


@pytest.mark.parametrize("name", sorted(CASES))
def test_ms_solve_fp64_follows_oracle(name):
    dwf = lib()
    p, U, phi, blk, l, ncol, n, xo, hist = case(name)
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_ms_solve(h, blk, l, "f64", ncol, cuda(phi), x, 0.0, n, history=n + 2,
                          raise_on_fail=False)
    assert st["status"] == dwf.DWF_ERR_NOT_CONVERGED and st["iterations"] == n
    for k in range(n):
        assert abs(st["history"][k] - hist[k + 1]) <= 1e-6 * hist[k + 1], (k, st["history"],
                                                                         hist)
    assert rel(host(x), xo) <= 1e-9
    assert st["operator_applications"] == n * ncol


@pytest.mark.parametrize("name", ["additive_mobius", "sap2_mobius"])
def test_ms_solve_fp16_local_solves(name):
    dwf = lib()
    p, U, phi, blk, l, ncol, n, xo, hist = case(name)
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_ms_solve(h, blk, l, "f16", ncol, cuda(phi), x, 0.0, n, history=n + 2,
                          raise_on_fail=False)
    res = o.true_residual(U, host(x), phi, p)
    assert abs(res - hist[-1]) <= 0.05 * hist[-1], (res, hist[-1])
    assert abs(st["true_residual"] - res) <= 1e-9


def test_ms_solve_argument_errors():
    dwf = lib()
    dims, Ls = (12, 4, 4, 4), 4
    h = dwf.dwf_create(dims, Ls, 1.8, 0.1, 1.0, 0.0, cuda(inputs.unit_links(dims)))
    phi = cuda(np.ones((Ls, 12 * 4 * 4 * 4 // 2, 4, 3), complex))
    x = cuda(np.zeros((Ls, 12 * 4 * 4 * 4 // 2, 4, 3), complex))
    for blk, ncol in (((4, 4, 4, 4), 2), ((4, 4, 4, 4), 16), ((2, 2, 2, 2), 3)):
        with pytest.raises(dwf.DWFError) as e:
            dwf.dwf_ms_solve(h, blk, 2, "f64", ncol, phi, x, 1e-8, 10)
        assert e.value.status == dwf.DWF_ERR_ARG
