"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle's tests.

This module only draws random numbers and arranges them into arrays: gauge links,
pseudofermion sources, random gauge transformations, su(3) directions and the list of
batched problems.  It holds none of the solver's arithmetic (no Dirac operator, no CG).

Recipe (the paper runs on a physical-pion-mass 32^3x64 ensemble that is not available;
these smooth synthetic fields stand in for it):

* generator: ``numpy.random.default_rng(seed)`` (PCG64);
* links: for every (t, z, y, x, mu) a 3x3 complex Gaussian matrix A (real parts for the whole
  field drawn first, then imaginary parts, both N(0,1)), H = (A + A^dag)/2 - tr(.)/3,
  U = V diag(exp(i eps lambda)) V^dag from the eigen-decomposition of H, so det U = 1;
* sources: complex Gaussian with E|z|^2 = 1 on even sites, shape [Ls][V/2][4][3]
  (even sites in lexicographic order, x fastest), drawn after the links from the same
  generator.

Layouts follow the C-ABI: links ``[T][Z][Y][X][mu][3][3]`` complex128 with mu = x, y, z, t;
dims are given as (X, Y, Z, T).
"""
from __future__ import annotations

import numpy as np

# Named synthetic workloads.  dims = (X, Y, Z, T).
CONFIGS = {
    # Shamir 4^4 x Ls=8: plain FP64 CG on the even-odd normal equations.
    "shamir_4x4x4x4_ls8": dict(dims=(4, 4, 4, 4), Ls=8, M5=1.8, mf=0.1, b=1.0, c=0.0,
                               eps=0.2, seed=1),
    # Shamir 16^4 x Ls=16: plain FP64 CG vs FP64 MSPCG with 2^4 blocks of 8^4, l = 6.
    "shamir_16x16x16x16_ls16": dict(dims=(16, 16, 16, 16), Ls=16, M5=1.8, mf=0.01, b=1.0,
                                    c=0.0, eps=0.3, seed=2, block=(8, 8, 8, 8), inner=6),
    # Moebius 24^3x48 x Ls=12: mixed FP16/FP32/FP64 MSPCG, 512 blocks of 6^4.
    "mobius_24x24x24x48_ls12": dict(dims=(24, 24, 24, 48), Ls=12, M5=1.8, mf=0.005, b=1.5,
                                    c=0.5, eps=0.35, seed=3, block=(6, 6, 6, 6), inner=6),
    # Force / differentiation workloads.
    "mobius_8x8x8x16_ls8": dict(dims=(8, 8, 8, 16), Ls=8, M5=1.8, mf=0.02, b=1.5, c=0.5,
                                eps=0.3, seed=5),
    "mobius_16x16x16x16_ls16": dict(dims=(16, 16, 16, 16), Ls=16, M5=1.8, mf=0.02, b=1.5,
                                    c=0.5, eps=0.3, seed=5),
}

# Batched workload: lattice and Ls choices of the 64 uneven Moebius problems.
BATCH_LATTICES = ((8, 8, 8, 8), (8, 8, 8, 16), (12, 12, 12, 12), (16, 16, 16, 32))
BATCH_LS = (8, 12, 16)


def _hermitian_traceless(a: np.ndarray) -> np.ndarray:
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1) / 3.0
    return h - tr[..., None, None] * np.eye(3)


def _exp_i(h: np.ndarray, eps: float) -> np.ndarray:
    lam, v = np.linalg.eigh(h)
    return (v * np.exp(1j * eps * lam)[..., None, :]) @ np.conj(np.swapaxes(v, -1, -2))


def random_su3(rng: np.random.Generator, shape: tuple, eps: float) -> np.ndarray:
    """SU(3) matrices U = exp(i eps H), H traceless Hermitian built from Gaussian entries."""
    shape = tuple(shape) + (3, 3)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return _exp_i(_hermitian_traceless(a), eps)


def gauge_links(dims, eps: float, rng: np.random.Generator) -> np.ndarray:
    """Links [T][Z][Y][X][4][3][3] complex128 (mu = x, y, z, t)."""
    X, Y, Z, T = dims
    return np.ascontiguousarray(random_su3(rng, (T, Z, Y, X, 4), eps))


def unit_links(dims) -> np.ndarray:
    X, Y, Z, T = dims
    u = np.zeros((T, Z, Y, X, 4, 3, 3), dtype=np.complex128)
    u[..., :, :] = np.eye(3)
    return u


def even_source(dims, Ls: int, rng: np.random.Generator) -> np.ndarray:
    """Complex Gaussian even-site source [Ls][V/2][4][3] with E|z|^2 = 1."""
    X, Y, Z, T = dims
    shape = (Ls, X * Y * Z * T // 2, 4, 3)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return np.ascontiguousarray((re + 1j * im) / np.sqrt(2.0))


def full_source(dims, Ls: int, rng: np.random.Generator) -> np.ndarray:
    """Complex Gaussian field on all sites [Ls][V][4][3] (lexicographic, x fastest)."""
    X, Y, Z, T = dims
    shape = (Ls, X * Y * Z * T, 4, 3)
    return np.ascontiguousarray(
        (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0))


def gauge_transform(dims, rng: np.random.Generator) -> np.ndarray:
    """Random SU(3) gauge transformation g(x), shape [T][Z][Y][X][3][3]."""
    X, Y, Z, T = dims
    return random_su3(rng, (T, Z, Y, X), 1.0)


def su3_directions(dims, rng: np.random.Generator) -> np.ndarray:
    """Random su(3) direction per link: Omega = sum_a w_a T_a, w_a ~ N(0,1), T_a = lambda_a/2.

    Returned as Hermitian traceless matrices [T][Z][Y][X][4][3][3].
    """
    X, Y, Z, T = dims
    w = rng.standard_normal((T, Z, Y, X, 4, 8))
    return np.einsum("...a,aij->...ij", w, gell_mann() / 2.0)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_a (a = 1..8), shape (8, 3, 3)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0, 0, 1] = l[0, 1, 0] = 1
    l[1, 0, 1], l[1, 1, 0] = -1j, 1j
    l[2, 0, 0], l[2, 1, 1] = 1, -1
    l[3, 0, 2] = l[3, 2, 0] = 1
    l[4, 0, 2], l[4, 2, 0] = -1j, 1j
    l[5, 1, 2] = l[5, 2, 1] = 1
    l[6, 1, 2], l[6, 2, 1] = -1j, 1j
    l[7, 0, 0] = l[7, 1, 1] = 1 / np.sqrt(3)
    l[7, 2, 2] = -2 / np.sqrt(3)
    return l


def workload(name: str, with_links: bool = True) -> dict:
    """Links and source of a named configuration, drawn in the documented order."""
    cfg = dict(CONFIGS[name])
    rng = np.random.default_rng(cfg["seed"])
    out = dict(cfg)
    out["name"] = name
    links = gauge_links(cfg["dims"], cfg["eps"], rng)
    out["links"] = links if with_links else None
    out["phi"] = even_source(cfg["dims"], cfg["Ls"], rng)
    return out


def batch_problems(n: int = 64, seed: int = 4) -> list:
    """Parameters of n independent Moebius problems (lattice, Ls, mf, eps, per-problem seed).

    Draw order per problem i: lattice index, Ls index, mf ~ U[0.005, 0.05], eps ~ U[0.2, 0.4];
    links and source then come from ``SeedSequence(seed).spawn(n)[i]``.
    """
    rng = np.random.default_rng(seed)
    children = np.random.SeedSequence(seed).spawn(n)
    probs = []
    for i in range(n):
        li = int(rng.integers(len(BATCH_LATTICES)))
        si = int(rng.integers(len(BATCH_LS)))
        mf = float(rng.uniform(0.005, 0.05))
        eps = float(rng.uniform(0.2, 0.4))
        probs.append(dict(dims=BATCH_LATTICES[li], Ls=BATCH_LS[si], mf=mf, eps=eps, M5=1.8,
                          b=1.5, c=0.5, seed_seq=children[i]))
    return probs


def batch_problem_fields(prob: dict):
    rng = np.random.default_rng(prob["seed_seq"])
    links = gauge_links(prob["dims"], prob["eps"], rng)
    phi = even_source(prob["dims"], prob["Ls"], rng)
    return links, phi
