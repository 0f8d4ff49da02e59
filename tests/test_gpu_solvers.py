"""GPU parity of the solvers (dwf_cg, dwf_mspcg) against the FP64 oracle.

FP64 CG and FP64 MSPCG follow the oracle's iteration step by step, so their iteration counts
must agree (to one step: the stopping test compares a residual that differs by rounding) and
their solutions must agree with the oracle's to 1e-9 at outer residual 1e-10.  Mixed-precision
solvers must reach the FP64 true residual 1e-10; their solution error against the oracle is
bounded by the conditioning (||e||/||x|| <= kappa ||r||/||b||) and reported."""
import numpy as np
import pytest

from oracle import dwf_oracle as o
from paper_1804_08593_gb300 import inputs
from tests.gpu_common import cuda, host, lib, rel

pytestmark = pytest.mark.gpu

_cache = {}


def c1():
    """Shamir 4^4 x 8 (M5 = 1.8, mf = 0.1, eps = 0.2, seed 1) and its oracle CG solution."""
    if "c1" not in _cache:
        w = inputs.workload("shamir_4x4x4x4_ls8")
        p = o.DWFParams(w["dims"], w["Ls"], w["M5"], w["mf"], w["b"], w["c"])
        U, phi = w["links"], w["phi"]
        x, k, hist = o.cg(lambda v: o.mdagm(U, v, p), phi, 1e-10, 5000)
        _cache["c1"] = (p, U, phi, x, k, hist)
    return _cache["c1"]


def small_ms():
    """Moebius 4^4 x 4, heavier mass: oracle MSPCG with 2^4 blocks in a few seconds."""
    if "ms" not in _cache:
        dims = (4, 4, 4, 4)
        rng = np.random.default_rng(21)
        p = o.DWFParams(dims, 4, 1.8, 0.3, 1.5, 0.5)
        U = inputs.gauge_links(dims, 0.2, rng)
        phi = inputs.even_source(dims, 4, rng)
        x, k, hist = o.mspcg(U, phi, p, (2, 2, 2, 2), 3, 1e-10, 500)
        _cache["ms"] = (p, U, phi, x, k, hist)
    return _cache["ms"]


def test_cg_fp64_matches_oracle():
    dwf = lib()
    p, U, phi, xo, ko, _ = c1()
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_cg(h, cuda(phi), x, 1e-10, 5000, "f64", history=6000)
    assert abs(st["iterations"] - ko) <= 1, (st["iterations"], ko)
    assert st["true_residual"] <= 1e-10
    assert rel(host(x), xo) <= 1e-9
    assert o.true_residual(U, host(x), phi, p) <= 1e-10
    assert len(st["history"]) == st["iterations"]


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_cg_mixed_precision_reliable_updates(prec):
    dwf = lib()
    p, U, phi, xo, ko, _ = c1()
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_cg(h, cuda(phi), x, 1e-10, 20000, prec)
    assert st["true_residual"] <= 1e-10
    assert st["reliable_updates"] >= 1
    assert o.true_residual(U, host(x), phi, p) <= 1.5e-10
    # error against the oracle's solution: conditioning-bounded, C1 is well conditioned
    assert rel(host(x), xo) <= 1e-7


def test_cg_bf16_reliable_updates_well_conditioned():
    """16-bit CG corrections only reduce the FP64 residual when kappa(A) * eps is below one
    (BF16: eps = 2^-8); on a heavy-mass problem BF16 CG with FP64 reliable updates reaches
    1e-10."""
    dwf = lib()
    dims, Ls = (4, 4, 4, 4), 8
    rng = np.random.default_rng(24)
    p = o.DWFParams(dims, Ls, 1.8, 0.8, 1.0, 0.0)
    U = inputs.gauge_links(dims, 0.2, rng)
    phi = inputs.even_source(dims, Ls, rng)
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_cg(h, cuda(phi), x, 1e-10, 5000, "bf16")
    assert st["true_residual"] <= 1e-10 and st["reliable_updates"] >= 2
    assert o.true_residual(U, host(x), phi, p) <= 1.5e-10


def test_cg_initial_guess_is_a_restart():
    dwf = lib()
    p, U, phi, xo, ko, _ = c1()
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(0.99 * xo)
    st = dwf.dwf_cg(h, cuda(phi), x, 1e-10, 5000, "f64")
    assert st["iterations"] < ko
    assert o.true_residual(U, host(x), phi, p) <= 1e-10


def test_cg_failure_modes():
    dwf = lib()
    p, U, phi, xo, ko, _ = c1()
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_cg(h, cuda(phi), x, 1e-10, 3, "f64", raise_on_fail=False)
    assert st["status"] == dwf.DWF_ERR_NOT_CONVERGED and st["iterations"] == 3
    bad = phi.copy()
    bad[0, 0, 0, 0] = np.nan
    with pytest.raises(dwf.DWFError) as e:
        dwf.dwf_cg(h, cuda(bad), cuda(np.zeros_like(phi)), 1e-10, 100, "f64")
    assert e.value.status == dwf.DWF_ERR_BREAKDOWN
    z = cuda(np.ones_like(phi))
    st = dwf.dwf_cg(h, cuda(np.zeros_like(phi)), z, 1e-10, 100, "f64")
    assert np.all(host(z) == 0)


@pytest.mark.parametrize("solver", ["persistent", "stages"])
def test_mspcg_fp64_matches_oracle(solver, monkeypatch):
    monkeypatch.setenv("DWF_LOCAL_SOLVER", solver)
    dwf = lib()
    p, U, phi, xo, ko, hist = small_ms()
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_mspcg(h, (2, 2, 2, 2), 3, "f64", "f64", cuda(phi), x, 1e-10, 500, history=600)
    assert abs(st["iterations"] - ko) <= 1, (st["iterations"], ko)
    # residual history follows the oracle's step by step
    n = min(len(st["history"]), len(hist) - 1)
    for k in range(n):
        assert abs(st["history"][k] - hist[k + 1]) <= 1e-6 * hist[k + 1] + 1e-13
    assert st["true_residual"] <= 1e-10
    assert rel(host(x), xo) <= 1e-9


def test_mspcg_flexible_fp64():
    dwf = lib()
    p, U, phi, xo, ko, _ = small_ms()
    xf, kf, _ = o.mspcg(U, phi, p, (2, 2, 2, 2), 3, 1e-10, 500, flexible=True)
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_mspcg(h, (2, 2, 2, 2), 3, "f64", "f64", cuda(phi), x, 1e-10, 500,
                       flexible=True)
    assert abs(st["iterations"] - kf) <= 1
    assert rel(host(x), xf) <= 1e-9


@pytest.mark.parametrize("inner", ["f16", "bf16", "f32"])
def test_mspcg_mixed_precision(inner):
    dwf = lib()
    p, U, phi, xo, ko, _ = c1()
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_mspcg(h, (2, 2, 2, 2), 6, inner, "f32", cuda(phi), x, 1e-10, 2000)
    assert st["true_residual"] <= 1e-10
    assert o.true_residual(U, host(x), phi, p) <= 1.5e-10
    assert rel(host(x), xo) <= 1e-7
    # the initial preconditioning plus one per outer iteration but the converged one
    assert st["inner_iterations"] == 6 * st["iterations"]


def test_mspcg_single_block_many_local_iterations():
    """One block = the whole lattice with many local iterations: M^-1 ~ A^-1, so the outer
    iteration converges in very few steps (exact-preconditioner limit of Sec. 2.3)."""
    dwf = lib()
    p, U, phi, xo, ko, _ = small_ms()
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_mspcg(h, p.dims, 200, "f64", "f64", cuda(phi), x, 1e-10, 50)
    assert st["iterations"] <= 2
    assert rel(host(x), xo) <= 1e-9


def exact_case():
    """Shamir 8x4x2x2 x 4 with two 4x4x2x2 blocks: the exact block preconditioner cuts the
    global iteration count by more than 2 (oracle: CG 128, MSPCG 56)."""
    if "ex" not in _cache:
        dims = (8, 4, 2, 2)
        rng = np.random.default_rng(3)
        p = o.DWFParams(dims, 4, 1.8, 0.1, 1.0, 0.0)
        U = inputs.gauge_links(dims, 0.2, rng)
        phi = inputs.even_source(dims, 4, rng)
        x, k, hist = o.mspcg(U, phi, p, (4, 4, 2, 2), 6, 1e-10, 500, local_op="exact")
        _cache["ex"] = (p, U, phi, x, k, hist)
    return _cache["ex"]


@pytest.mark.parametrize("solver", ["persistent", "stages"])
def test_mspcg_exact_blocks_fp64_matches_oracle(solver, monkeypatch):
    monkeypatch.setenv("DWF_LOCAL_SOLVER", solver)
    dwf = lib()
    p, U, phi, xo, ko, hist = exact_case()
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_mspcg(h, (4, 4, 2, 2), 6, "f64", "f64", cuda(phi), x, 1e-10, 500,
                       local_op=dwf.LOCAL_EXACT, history=600)
    assert abs(st["iterations"] - ko) <= 1, (st["iterations"], ko)
    n = min(len(st["history"]), len(hist) - 1)
    for k in range(n):
        assert abs(st["history"][k] - hist[k + 1]) <= 1e-6 * hist[k + 1] + 1e-13
    assert rel(host(x), xo) <= 1e-9


def test_mspcg_exact_blocks_moebius_many_blocks():
    """Moebius 4x4x4x2 x 4 with eight 2x2x2x2 blocks (halos wrap around the lattice)."""
    dwf = lib()
    dims = (4, 4, 4, 2)
    rng = np.random.default_rng(23)
    p = o.DWFParams(dims, 4, 1.8, 0.3, 1.5, 0.5)
    U = inputs.gauge_links(dims, 0.3, rng)
    phi = inputs.even_source(dims, 4, rng)
    xo, ko, hist = o.mspcg(U, phi, p, (2, 2, 2, 2), 3, 1e-10, 500, local_op="exact")
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_mspcg(h, (2, 2, 2, 2), 3, "f64", "f64", cuda(phi), x, 1e-10, 500,
                       local_op=dwf.LOCAL_EXACT, history=600)
    assert abs(st["iterations"] - ko) <= 1, (st["iterations"], ko)
    assert rel(host(x), xo) <= 1e-9


@pytest.mark.parametrize("inner", ["f16", "bf16"])
def test_mspcg_exact_blocks_mixed_precision(inner):
    dwf = lib()
    p, U, phi, xo, ko, _ = c1()
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_mspcg(h, (2, 2, 2, 2), 6, inner, "f32", cuda(phi), x, 1e-10, 2000,
                       local_op=dwf.LOCAL_EXACT)
    assert st["true_residual"] <= 1e-10
    assert o.true_residual(U, host(x), phi, p) <= 1.5e-10
    assert rel(host(x), xo) <= 1e-7


@pytest.mark.parametrize("solver", ["cg_f64", "cg_f32", "mspcg"])
def test_zero_source_gives_zero_solution(solver):
    """phi = 0: every solver returns x = 0 at once (no division by a zero norm)."""
    dwf = lib()
    p, U, phi, _, _, _ = c1()
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    z = cuda(np.zeros_like(phi))
    x = cuda(np.ones_like(phi))
    if solver == "mspcg":
        st = dwf.dwf_mspcg(h, (2, 2, 2, 2), 2, "f16", "f32", z, x, 1e-10, 100)
    else:
        st = dwf.dwf_cg(h, z, x, 1e-10, 100, solver[3:])
    assert st["iterations"] == 0
    assert np.count_nonzero(host(x)) == 0


# ---------------------------------------------------------------------------------------
# The exact block operator P_s A P_s at block shapes that span several 32-site tiles and have
# interior sites: 6^4 blocks (648 even sites = 21 tiles, the benchmark workload's block
# shape) and 8^4 blocks.  FP64 MSPCG must follow the oracle step by step; the comparison runs
# a fixed number of outer iterations (maxit) so the oracle finishes in seconds.
# ---------------------------------------------------------------------------------------
MULTI_TILE = {
    # name: dims, Ls, block, (b, c), mf, local iterations l, outer iterations, seed
    "shamir_12x12x6x6_ls4_b6": ((12, 12, 6, 6), 4, (6, 6, 6, 6), (1.0, 0.0), 0.1, 2, 6, 31),
    "mobius_12x6x6x6_ls8_b6": ((12, 6, 6, 6), 8, (6, 6, 6, 6), (1.5, 0.5), 0.05, 3, 6, 32),
    "shamir_16x8x8x8_ls4_b8": ((16, 8, 8, 8), 4, (8, 8, 8, 8), (1.0, 0.0), 0.1, 2, 5, 33),
}


def multi_tile(name):
    if name not in _cache:
        dims, Ls, blk, (b, c), mf, l, n, seed = MULTI_TILE[name]
        rng = np.random.default_rng(seed)
        p = o.DWFParams(dims, Ls, 1.8, mf, b, c)
        U = inputs.gauge_links(dims, 0.3, rng)
        phi = inputs.even_source(dims, Ls, rng)
        _cache[name] = (p, U, phi, blk, l, n)
    return _cache[name]


def multi_tile_oracle(name):
    key = name + "/oracle"
    if key not in _cache:
        p, U, phi, blk, l, n = multi_tile(name)
        _cache[key] = o.mspcg(U, phi, p, blk, l, 1e-14, n, local_op="exact")
    return _cache[key]


@pytest.mark.parametrize("solver", ["persistent", "stages"])
@pytest.mark.parametrize("name", sorted(MULTI_TILE))
def test_mspcg_exact_multi_tile_blocks_follow_oracle(name, solver, monkeypatch):
    """Both local-solve implementations (one persistent launch; one launch per stage)."""
    monkeypatch.setenv("DWF_LOCAL_SOLVER", solver)
    dwf = lib()
    p, U, phi, blk, l, n = multi_tile(name)
    xo, ko, hist = multi_tile_oracle(name)
    assert ko == n
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_mspcg(h, blk, l, "f64", "f64", cuda(phi), x, 1e-14, n,
                       local_op=dwf.LOCAL_EXACT, history=n + 4, raise_on_fail=False)
    assert st["status"] == dwf.DWF_ERR_NOT_CONVERGED and st["iterations"] == n
    for k in range(n):
        assert abs(st["history"][k] - hist[k + 1]) <= 1e-6 * hist[k + 1], (k, st["history"][k],
                                                                         hist[k + 1])
    assert rel(host(x), xo) <= 1e-9


@pytest.mark.parametrize("inner", ["f16", "bf16"])
@pytest.mark.parametrize("name", ["shamir_12x12x6x6_ls4_b6", "mobius_12x6x6x6_ls8_b6"])
def test_mspcg_mixed_multi_tile_blocks_true_residual(name, inner):
    """16-bit local solves, FP32 outer CG, FP64 reliable updates on the multi-tile blocks:
    the oracle recomputes the true residual of the returned solution."""
    dwf = lib()
    p, U, phi, blk, l, n = multi_tile(name)
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_mspcg(h, blk, l, inner, "f32", cuda(phi), x, 1e-10, 5000,
                       local_op=dwf.LOCAL_EXACT)
    assert st["true_residual"] <= 1e-10
    assert o.true_residual(U, host(x), phi, p) <= 1.5e-10


@pytest.mark.parametrize("flexible", [False, True])
def test_mspcg_preconditioner_graph_replays_the_direct_launches(flexible, monkeypatch):
    """The preconditioner step of the persistent local solver is captured in a CUDA graph once
    its launch variant is fixed (forced here, so from the first call) and replayed on every
    later call of a handle with its own stream: the solve must be bit for bit the one the
    direct launches give, and reach the oracle-recomputed true residual."""
    import torch
    monkeypatch.setenv("DWF_LOCAL_VARIANT", "0")
    dwf = lib()
    p, U, phi, blk, l, n = multi_tile("mobius_12x6x6x6_ls8_b6")
    stream = torch.cuda.Stream()   # the legacy default stream cannot be captured
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U), stream)
    out = {}
    for graph in ("1", "0"):
        monkeypatch.setenv("DWF_PRECOND_GRAPH", graph)
        x = cuda(np.zeros_like(phi))
        st = dwf.dwf_mspcg(h, blk, l, "f16", "f32", cuda(phi), x, 1e-10, 5000,
                           local_op=dwf.LOCAL_EXACT, flexible=flexible, history=5000)
        out[graph] = (st, host(x))
    (sg, xg), (sd, xd) = out["1"], out["0"]
    assert sg["iterations"] == sd["iterations"] and sg["iterations"] > 2
    assert sg["history"] == sd["history"]
    assert np.array_equal(xg, xd)
    assert o.true_residual(U, xg, phi, p) <= 1.5e-10


def test_cg_lanczos_kappa_matches_dense_spectrum():
    """The CG coefficients recorded by dwf_cg (residual norms and curvatures <p, A p>) give
    the Lanczos tridiagonal of A; its extreme eigenvalues are those of the dense A built by
    the oracle on a 2^4 x 4 lattice."""
    import bench
    dwf = lib()
    dims, Ls = (2, 2, 2, 2), 4
    rng = np.random.default_rng(61)
    p = o.DWFParams(dims, Ls, 1.8, 0.2, 1.5, 0.5)
    U = inputs.gauge_links(dims, 0.3, rng)
    phi = inputs.even_source(dims, Ls, rng)
    n = phi.size
    A = np.zeros((n, n), complex)
    for j in range(n):
        e = np.zeros(n, complex)
        e[j] = 1.0
        A[:, j] = o.mdagm(U, e.reshape(phi.shape), p).reshape(-1)
    ev = np.linalg.eigvalsh((A + A.conj().T) / 2)
    h = dwf.dwf_create(dims, Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(np.zeros_like(phi))
    st = dwf.dwf_cg(h, cuda(phi), x, 1e-13, 2000, "f64", history=2000, curvature=True)
    kappa, lmin, lmax = bench.lanczos_kappa(st["history"], st["curvature_history"])
    assert abs(lmax - ev[-1]) <= 1e-8 * ev[-1]
    assert abs(lmin - ev[0]) <= 1e-4 * ev[0]
    assert abs(kappa - ev[-1] / ev[0]) <= 1e-4 * kappa
