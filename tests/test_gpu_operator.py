"""GPU parity of the operator stages (dwf_apply) against the FP64 oracle, element by element.

Tolerances (relative L2 error of one application, same FP64 input): FP64 1e-13, FP32 1e-6,
FP16/BF16 5e-3 (input rounding included).  Lattices span several 32-site tiles and include a
ragged tail (V/2 not a multiple of 32)."""
import numpy as np
import pytest

from oracle import dwf_oracle as o
from paper_1804_08593_gb300 import inputs
from tests.gpu_common import TOL, cuda, host, lib, rand_even, rand_full, rel

pytestmark = pytest.mark.gpu

CASES = [
    # dims, Ls, M5, mf, b, c, eps
    ((2, 2, 2, 2), 4, 1.8, 0.1, 1.0, 0.0, 0.4),      # tiny, one partial tile
    ((4, 6, 2, 6), 6, 1.8, 0.05, 1.5, 0.5, 0.3),     # 144 even sites: ragged tail
    ((4, 4, 4, 4), 8, 1.8, 0.1, 1.0, 0.0, 0.2),      # Shamir 4^4 x 8
    ((8, 8, 8, 16), 8, 1.8, 0.02, 1.5, 0.5, 0.3),    # Moebius 8^3x16 x 8, many tiles
    ((4, 4, 4, 8), 12, 1.8, 0.005, 1.5, 0.5, 0.35),  # Ls = 12 Moebius
    ((4, 4, 4, 4), 16, 1.8, 0.01, 1.0, 0.0, 0.3),    # Ls = 16 Shamir
    ((4, 4, 2, 2), 10, 1.6, 0.2, 2.0, 1.0, 0.5),     # Ls = 10, b - c != 1... general b, c
    ((4, 4, 2, 4), 8, 1.8, 0.1, 1.25, 0.0, 0.3),     # c = 0, b != 1: D+ = b absorbed
    ((4, 2, 4, 4), 6, 1.8, 0.1, 0.5, 1.5, 0.3),      # |beta/alpha| > 1: matrices only
    ((4, 2, 2, 4), 4, 1.8, 1.0, 1.5, 0.5, 0.3),      # mf = 1: the walls close without sign change
]


def _setup(case, seed=0):
    dims, Ls, M5, mf, b, c, eps = case
    rng = np.random.default_rng(seed)
    U = inputs.gauge_links(dims, eps, rng)
    p = o.DWFParams(dims, Ls, M5, mf, b, c)
    return rng, U, p


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_even_odd_operators(case, prec):
    dwf = lib()
    rng, U, p = _setup(case)
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = rand_even(rng, p.dims, p.Ls)
    dx = cuda(x)
    out = cuda(np.zeros_like(x))
    for op, ref in (("Mpc", o.mpc(U, x, p)), ("Mpc_dag", o.mpc_dag(U, x, p)),
                    ("MdagM", o.mdagm(U, x, p))):
        dwf.dwf_apply(h, op, dx, out, prec)
        err = rel(host(out), ref)
        assert err <= TOL[prec], (op, prec, err)


@pytest.mark.parametrize("case", CASES[:5])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_full_operator(case, prec):
    dwf = lib()
    rng, U, p = _setup(case, 1)
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    X, Y, Z, T = p.dims
    psi = rand_full(rng, p.dims, p.Ls)
    out = cuda(np.zeros_like(psi))
    shape5 = (p.Ls, T, Z, Y, X, 4, 3)
    for op, dag in (("M", False), ("Mdag", True)):
        dwf.dwf_apply(h, op, cuda(psi), out, prec)
        ref = o.dwf(U, psi.reshape(shape5), p, dag=dag).reshape(psi.shape)
        assert rel(host(out), ref) <= TOL[prec], (op, prec)


def test_host_buffers_match_device_buffers():
    dwf = lib()
    rng, U, p = _setup(CASES[3], 2)
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, U)       # host links
    x = rand_even(rng, p.dims, p.Ls)
    out_h = np.zeros_like(x)
    dwf.dwf_apply(h, "MdagM", x, out_h, "f64")                        # host in/out
    out_d = cuda(np.zeros_like(x))
    dwf.dwf_apply(h, "MdagM", cuda(x), out_d, "f64")
    assert np.array_equal(out_h, host(out_d))
    assert rel(out_h, o.mdagm(U, x, p)) <= 1e-13


def test_update_links_and_free_field():
    """U = 1 after an update: the operator follows the new links (free-field plane wave)."""
    dwf = lib()
    dims, Ls = (4, 4, 4, 8), 4
    rng, U, p = _setup(((4, 4, 4, 8), 4, 1.8, 0.1, 1.5, 0.5, 0.3), 3)
    h = dwf.dwf_create(dims, Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    U1 = inputs.unit_links(dims)
    dwf.dwf_update_links(h, cuda(U1))
    x = rand_even(rng, dims, Ls)
    out = cuda(np.zeros_like(x))
    dwf.dwf_apply(h, "MdagM", cuda(x), out, "f64")
    assert rel(host(out), o.mdagm(U1, x, p)) <= 1e-13


def test_deterministic_repeat():
    """Two applications give bit-identical results (no atomics in the data path)."""
    dwf = lib()
    rng, U, p = _setup(CASES[3], 4)
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(rand_even(rng, p.dims, p.Ls))
    a, b = cuda(np.zeros(x.shape, complex)), cuda(np.zeros(x.shape, complex))
    dwf.dwf_apply(h, "MdagM", x, a, "f32")
    dwf.dwf_apply(h, "MdagM", x, b, "f32")
    assert np.array_equal(host(a), host(b))


def test_bad_arguments_raise():
    dwf = lib()
    rng, U, p = _setup(CASES[2], 5)
    with pytest.raises(dwf.DWFError):
        dwf.dwf_create((4, 4, 4, 3), 8, 1.8, 0.1, 1.0, 0.0, cuda(U))     # odd dim
    with pytest.raises(dwf.DWFError):
        dwf.dwf_create(p.dims, 7, 1.8, 0.1, 1.0, 0.0, cuda(U))          # unsupported Ls
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    x = cuda(rand_even(rng, p.dims, p.Ls))
    with pytest.raises(dwf.DWFError):
        dwf.dwf_apply(h, "MdagM", x, x, "f64")                          # aliasing
    with pytest.raises(dwf.DWFError):
        dwf.dwf_mspcg(h, (3, 4, 4, 4), 2, "f32", "f32", x, cuda(np.zeros(x.shape, complex)),
                      1e-8, 10)                                          # bad block


@pytest.mark.parametrize("case", [CASES[1], CASES[3], CASES[4], CASES[5]])
@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_tensor_core_m5_matches_cuda_core_path(case, prec, monkeypatch):
    """The FP16/BF16 stages apply the Ls x Ls fifth-dimension matrices with tcgen05 MMAs;
    DWF_DISABLE_TC=1 at handle creation selects the FP32 CUDA-core column GEMM instead.
    Both must meet the 16-bit operator tolerance against the oracle and agree closely."""
    dwf = lib()
    rng, U, p = _setup(case, 7)
    x = rand_even(rng, p.dims, p.Ls)
    ref = o.mdagm(U, x, p)
    outs = {}
    monkeypatch.setenv("DWF_POST", "matrix")   # no recurrence candidate: TC vs CUDA cores
    for flag in ("0", "1"):
        monkeypatch.setenv("DWF_DISABLE_TC", flag)
        h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
        out = cuda(np.zeros_like(x))
        dwf.dwf_apply(h, "MdagM", cuda(x), out, prec)
        outs[flag] = host(out)
        assert rel(outs[flag], ref) <= TOL[prec], (flag, rel(outs[flag], ref))
    # both round the result to the same 16-bit storage, so they agree to that precision
    assert rel(outs["0"], outs["1"]) <= TOL[prec]


@pytest.mark.parametrize("case", [CASES[1], CASES[2], CASES[4], CASES[6], CASES[7]])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("mode", ["matrix", "recurrence"])
def test_post_by_matrix_and_by_recurrence(case, prec, mode, monkeypatch):
    """D+ M5op^-1 and M5op^-dag D+^dag are applied either as dense Ls x Ls matrices or by the
    O(Ls) bidiagonal recurrences with the Sherman-Morrison wall correction (DWF_POST at
    handle creation).  Both must meet the operator tolerance for Mpc, Mpc^dag and MdagM."""
    dwf = lib()
    rng, U, p = _setup(case, 11)
    x = rand_even(rng, p.dims, p.Ls)
    monkeypatch.setenv("DWF_POST", mode)
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    for op, ref in (("Mpc", o.mpc(U, x, p)), ("Mpc_dag", o.mpc_dag(U, x, p)),
                    ("MdagM", o.mdagm(U, x, p))):
        out = cuda(np.zeros_like(x))
        dwf.dwf_apply(h, op, cuda(x), out, prec)
        assert rel(host(out), ref) <= TOL[prec], (op, rel(host(out), ref))


@pytest.mark.parametrize("variant", [str(i) for i in range(9)])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_every_launch_variant_matches_oracle(variant, prec, monkeypatch):
    """Every compiled launch variant of the stages (register budget, grid, link staging,
    neighbour gather, slices per thread), forced with DWF_STAGE_VARIANT, meets the operator
    tolerance on a lattice with a ragged tail, in the full and the dagger stages."""
    dwf = lib()
    rng, U, p = _setup(CASES[1], 13)
    x = rand_even(rng, p.dims, p.Ls)
    monkeypatch.setenv("DWF_STAGE_VARIANT", variant)
    h = dwf.dwf_create(p.dims, p.Ls, p.M5, p.mf, p.b, p.c, cuda(U))
    for op, ref in (("Mpc", o.mpc(U, x, p)), ("Mpc_dag", o.mpc_dag(U, x, p)),
                    ("MdagM", o.mdagm(U, x, p))):
        out = cuda(np.zeros_like(x))
        dwf.dwf_apply(h, op, cuda(x), out, prec)
        assert rel(host(out), ref) <= TOL[prec], (variant, op, rel(host(out), ref))
