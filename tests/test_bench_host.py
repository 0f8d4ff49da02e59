"""Host-side measurement logic of bench.py (no GPU)."""
import numpy as np

import bench


def _cg_coefficients(A, b, iters):
    """Plain CG from x = 0 recording ||r_{k+1}||/||b|| and <p_k, A p_k>/||b||^2."""
    bb = float(np.vdot(b, b).real)
    r = b.copy()
    p = r.copy()
    rr = bb
    res, curv = [], []
    for _ in range(iters):
        ap = A @ p
        pap = float(np.vdot(p, ap).real)
        alpha = rr / pap
        r = r - alpha * ap
        rr_new = float(np.vdot(r, r).real)
        p = r + (rr_new / rr) * p
        rr = rr_new
        res.append(np.sqrt(rr / bb))
        curv.append(pap / bb)
        if rr / bb < 1e-28:
            break
    return res, curv


def test_lanczos_kappa_recovers_extreme_eigenvalues():
    rng = np.random.default_rng(3)
    n = 120
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    ev = np.geomspace(0.01, 50.0, n)
    A = (Q * ev) @ Q.conj().T
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    res, curv = _cg_coefficients(A, b, 400)
    kappa, lmin, lmax = bench.lanczos_kappa(res, curv)
    assert abs(lmin - ev[0]) <= 1e-4 * ev[0]
    assert abs(lmax - ev[-1]) <= 1e-8 * ev[-1]
    assert abs(kappa - 5000.0) <= 1e-4 * 5000.0


def test_lanczos_kappa_first_step_is_rayleigh_quotient():
    """One CG step: T is 1x1 with entry 1/alpha_0 = <b, A b>/<b, b> (the Rayleigh quotient)."""
    rng = np.random.default_rng(4)
    n = 10
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    b = rng.standard_normal(n)
    res, curv = _cg_coefficients(A, b, 1)
    kappa, lmin, lmax = bench.lanczos_kappa(res, curv)
    rq = float(b @ A @ b / (b @ b))
    assert abs(lmin - rq) <= 1e-12 * rq and abs(lmax - rq) <= 1e-12 * rq and kappa == 1.0
