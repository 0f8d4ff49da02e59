"""GPU force and action (dwf_force, dwf_action, the autograd Function) against the oracle and
against FP64 central finite differences (h = 1e-5, random su(3) directions)."""
import numpy as np
import pytest

from oracle import dwf_oracle as o
from paper_1804_08593_gb300 import inputs
from tests.gpu_common import cuda, host, lib, rel

pytestmark = pytest.mark.gpu


def _case(dims, Ls, mf, b, c, eps, seed):
    rng = np.random.default_rng(seed)
    p = o.DWFParams(dims, Ls, 1.8, mf, b, c)
    U = inputs.gauge_links(dims, eps, rng)
    phi = inputs.even_source(dims, Ls, rng)
    return rng, p, U, phi


@pytest.mark.parametrize("prm", [((4, 4, 4, 4), 4, 0.1, 1.0, 0.0, 0.3, 31),
                                 ((4, 6, 2, 6), 6, 0.05, 1.5, 0.5, 0.3, 32),
                                 ((8, 8, 8, 16), 8, 0.02, 1.5, 0.5, 0.3, 5)])
def test_force_matches_oracle(prm):
    dwf = lib()
    rng, p, U, phi = _case(*prm)
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    X = cuda(np.zeros_like(phi))
    dwf.dwf_cg(h, cuda(phi), X, 1e-12, 100000, "f64")
    Xh = host(X)
    F = cuda(np.zeros_like(U))
    dwf.dwf_force(h, cuda(phi), X, F)
    Fo = o.force(U, phi, p, X=Xh)
    assert rel(host(F), Fo) <= 1e-12
    S = dwf.dwf_action(h, cuda(phi), X)
    So = o.action(U, phi, p, X=Xh)
    assert abs(S - So) <= 1e-12 * abs(So)


@pytest.mark.parametrize("name", ["mobius_8x8x8x16_ls8", "mobius_16x16x16x16_ls16"])
def test_force_central_differences(name):
    """Moebius 8^3x16 x Ls=8 and 16^4 x Ls=16 (mf = 0.02, eps = 0.3, seed 5): analytic gradient
    vs FP64 central differences of the action (stationary estimator, solves to 1e-13) along 20
    random su(3) directions, all links at once."""
    dwf = lib()
    w = inputs.workload(name)
    p = o.DWFParams(w["dims"], w["Ls"], w["M5"], w["mf"], w["b"], w["c"])
    U, phi = w["links"], w["phi"]
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    dphi = cuda(phi)

    def action(Uv):
        dwf.dwf_update_links(h, cuda(Uv))
        return dwf.dwf_action(h, dphi, None, tol=1e-13)

    dwf.dwf_update_links(h, cuda(U))
    F = cuda(np.zeros_like(U))
    dwf.dwf_force(h, dphi, None, F, tol=1e-13)
    F = host(F)
    rng = np.random.default_rng(5)
    hstep = 1e-5
    for _ in range(20):
        Om = inputs.su3_directions(p.dims, rng)
        lam, V = np.linalg.eigh(Om)

        def rot(t):
            return (V * np.exp(1j * t * lam)[..., None, :]) @ o.dagger(V) @ U

        fd = (action(rot(hstep)) - action(rot(-hstep))) / (2 * hstep)
        an = float(np.sum(np.real(np.conj(F) * (1j * Om @ U))))
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_autograd_function():
    torch = pytest.importorskip("torch")
    dwf = lib()
    from paper_1804_08593_gb300.autograd import pseudofermion_action
    rng, p, U, phi = _case((4, 4, 4, 4), 4, 0.1, 1.5, 0.5, 0.3, 33)
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    Ut = cuda(U).requires_grad_(True)
    S = pseudofermion_action(Ut, cuda(phi), h)
    S.backward()
    Fo = o.force(U, phi, p, tol=1e-13)
    assert rel(Ut.grad.cpu().numpy(), Fo) <= 1e-9
    So = o.action(U, phi, p, tol=1e-13)
    assert abs(float(S) - So) <= 1e-10 * abs(So)
