"""Shared helpers of the GPU parity tests: building the library, moving fields to the GPU,
and the relative-error measure used throughout."""
import numpy as np

from paper_1804_08593_gb300 import inputs

_built = False


def lib():
    """Builds (once) and loads libdwf; returns the binding module."""
    global _built
    if not _built:
        from paper_1804_08593_gb300 import build
        build.build()
        _built = True
    from paper_1804_08593_gb300 import dwf
    dwf.load()
    return dwf


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def rel(a, b):
    """||a - b||_2 / ||b||_2."""
    return float(np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1)))


def rand_even(rng, dims, Ls):
    X, Y, Z, T = dims
    s = (Ls, X * Y * Z * T // 2, 4, 3)
    return (rng.standard_normal(s) + 1j * rng.standard_normal(s)) / np.sqrt(2)


def rand_full(rng, dims, Ls):
    return inputs.full_source(dims, Ls, rng)


# Storage-precision tolerances of one operator application (relative L2 error).
TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 5e-3, "bf16": 5e-3}
