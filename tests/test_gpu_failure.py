"""Failure detection on the GPU without a fault: a bounded device-side wait that runs out.

With the handle's test switch DWF_OPT_TEST_WAIT_PROBE on, every FP32/FP16 operator stage runs
its TMA link-staging variant without issuing the copies, so the mbarrier it waits on can never
complete; the wait gives up after the handle's limit (DWF_OPT_WAIT_LIMIT_US), the kernel
returns, and the call reports DWF_ERR_TIMEOUT.  Nothing is left in flight, so the same handle
must then give correct results again (operator and a solver whose reductions the aborted
launch left unfinished)."""
import numpy as np
import pytest

from oracle import dwf_oracle as o
from paper_1804_08593_gb300 import inputs
from tests.gpu_common import TOL, cuda, host, lib, rand_even, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_wait_runs_out_then_handle_recovers(prec):
    dwf = lib()
    dims, Ls = (8, 8, 4, 8), 8
    rng = np.random.default_rng(51)
    p = o.DWFParams(dims, Ls, 1.8, 0.1, 1.5, 0.5)
    U = inputs.gauge_links(dims, 0.3, rng)
    x = rand_even(rng, dims, Ls)
    h = dwf.dwf_create(dims, Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    dx, out = cuda(x), cuda(np.zeros_like(x))
    dwf.dwf_set_option(h, dwf.OPT_WAIT_LIMIT_US, 200)
    dwf.dwf_set_option(h, dwf.OPT_TEST_WAIT_PROBE, 1)
    with pytest.raises(dwf.DWFError) as e:
        dwf.dwf_apply(h, "MdagM", dx, out, prec)
    assert e.value.status == dwf.DWF_ERR_TIMEOUT
    assert "gave up" in str(e.value)
    dwf.dwf_set_option(h, dwf.OPT_TEST_WAIT_PROBE, 0)
    dwf.dwf_apply(h, "MdagM", dx, out, prec)
    assert rel(host(out), o.mdagm(U, x, p)) <= TOL[prec]
    phi = inputs.even_source(dims, Ls, rng)
    xs = cuda(np.zeros_like(phi))
    st = dwf.dwf_cg(h, cuda(phi), xs, 1e-10, 20000, "f32")
    assert st["true_residual"] <= 1e-10
    assert o.true_residual(U, host(xs), phi, p) <= 1.5e-10


def test_options_reject_bad_values():
    dwf = lib()
    dims, Ls = (4, 4, 4, 4), 4
    h = dwf.dwf_create(dims, Ls, 1.8, 0.1, 1.0, 0.0, cuda(inputs.unit_links(dims)))
    for opt, val in ((dwf.OPT_WAIT_LIMIT_US, 0.0), (dwf.OPT_WAIT_LIMIT_US, 1e9), (7, 1.0)):
        with pytest.raises(dwf.DWFError) as e:
            dwf.dwf_set_option(h, opt, val)
        assert e.value.status == dwf.DWF_ERR_ARG
