"""Thin Python binding of libdwf.so (the C ABI declared in include/dwf.h).

Argument marshalling only: every step of every call runs in the library's CUDA kernels.
Fields are complex128 torch tensors (CUDA or CPU) or numpy arrays, in the layouts of the C
ABI: links [T][Z][Y][X][4][3][3], even-half fields [Ls][V/2][4][3], full fields [Ls][V][4][3].
The library must have been built (``paper_1804_08593_gb300.build.build()``); there is no
fallback implementation and a missing library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libdwf.so")

DWF_OK, DWF_ERR_ARG, DWF_ERR_CUDA, DWF_ERR_NOMEM = 0, 1, 2, 3
DWF_ERR_NOT_CONVERGED, DWF_ERR_BREAKDOWN, DWF_ERR_TIMEOUT = 4, 5, 6
F64, F32, F16, BF16 = 0, 1, 2, 3
PREC = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16}
OP_M, OP_MDAG, OP_MPC, OP_MPC_DAG, OP_MDAGM = 0, 1, 2, 3, 4
OPS = {"M": OP_M, "Mdag": OP_MDAG, "Mpc": OP_MPC, "Mpc_dag": OP_MPC_DAG, "MdagM": OP_MDAGM}
LOCAL_DROP, LOCAL_EXACT = 0, 1

# Every symbol include/dwf.h declares.
EXPORTS = ("dwf_create", "dwf_update_links", "dwf_apply", "dwf_cg", "dwf_mspcg", "dwf_force",
           "dwf_action", "dwf_batch_solve", "dwf_last_error", "dwf_destroy", "dwf_version",
           "dwf_profile_enable", "dwf_profile_read", "dwf_mdagm_noalloc", "dwf_set_option",
           "dwf_measure_peak", "dwf_ms_solve")
OPT_WAIT_LIMIT_US, OPT_TEST_WAIT_PROBE = 0, 1


class DWFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libdwf status {status}: {msg}")
        self.status = status


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("inner_iterations", ctypes.c_int),
                ("reliable_updates", ctypes.c_int), ("operator_applications", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("history", ctypes.POINTER(ctypes.c_double)), ("history_capacity", ctypes.c_int),
                ("history_len", ctypes.c_int),
                ("curvature_history", ctypes.POINTER(ctypes.c_double))]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_
             if k not in ("history", "curvature_history")}
        if self.history_len:
            d["history"] = [self.history[i] for i in range(self.history_len)]
            if self.curvature_history:
                d["curvature_history"] = [self.curvature_history[i]
                                          for i in range(self.history_len)]
        return d


class Problem(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("Ls", ctypes.c_int), ("M5", ctypes.c_double),
                ("mf", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double),
                ("links", ctypes.c_void_p), ("phi", ctypes.c_void_p), ("x", ctypes.c_void_p)]


class KernelProfile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int),
                ("ms_total", ctypes.c_double), ("bytes_total", ctypes.c_double),
                ("flops_total", ctypes.c_double)]


_lib = None


def load() -> ctypes.CDLL:
    """Loads libdwf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "paper_1804_08593_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.dwf_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(i), i, d, d, d, d, vp, vp]
    lib.dwf_update_links.argtypes = [vp, vp]
    lib.dwf_apply.argtypes = [vp, i, vp, vp, i]
    lib.dwf_cg.argtypes = [vp, vp, vp, d, i, i, ctypes.POINTER(Stats)]
    lib.dwf_mspcg.argtypes = [vp, ctypes.POINTER(i), i, i, i, i, i, vp, vp, d, i,
                              ctypes.POINTER(Stats)]
    lib.dwf_force.argtypes = [vp, vp, vp, vp, d]
    lib.dwf_action.argtypes = [vp, vp, vp, d, ctypes.POINTER(d)]
    lib.dwf_batch_solve.argtypes = [i, ctypes.POINTER(Problem), d, i, ctypes.POINTER(Stats), vp]
    lib.dwf_last_error.restype = ctypes.c_char_p
    lib.dwf_version.restype = ctypes.c_char_p
    lib.dwf_destroy.argtypes = [vp]
    lib.dwf_profile_enable.argtypes = [vp, i]
    lib.dwf_mdagm_noalloc.argtypes = [ctypes.POINTER(i), i, d, d, d, d, vp, vp, vp, i, vp]
    lib.dwf_profile_read.argtypes = [vp, ctypes.POINTER(KernelProfile), i, ctypes.POINTER(i)]
    lib.dwf_set_option.argtypes = [vp, i, d]
    lib.dwf_ms_solve.argtypes = [vp, ctypes.POINTER(i), i, i, i, i, vp, vp, d, i,
                                 ctypes.POINTER(Stats)]
    lib.dwf_measure_peak.argtypes = [i, vp, ctypes.POINTER(d)]
    for name in ("dwf_create", "dwf_update_links", "dwf_apply", "dwf_cg", "dwf_mspcg",
                 "dwf_force", "dwf_action", "dwf_batch_solve", "dwf_profile_enable",
                 "dwf_profile_read", "dwf_mdagm_noalloc", "dwf_set_option",
                 "dwf_measure_peak", "dwf_ms_solve"):
        getattr(lib, name).restype = i
    _lib = lib
    return lib


def dwf_last_error() -> str:
    return load().dwf_last_error().decode()


def dwf_version() -> str:
    return load().dwf_version().decode()


def _check(st: int, allow=()):
    if st != DWF_OK and st not in allow:
        raise DWFError(st, dwf_last_error())
    return st


def _ptr(t) -> int:
    """Address of a contiguous complex128 torch tensor or numpy array."""
    if isinstance(t, np.ndarray):
        if t.dtype != np.complex128 or not t.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous complex128")
        return t.ctypes.data
    import torch
    if t.dtype != torch.complex128 or not t.is_contiguous():
        raise ValueError("tensors must be contiguous complex128")
    return t.data_ptr()


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream or None
        except Exception:
            return None
        return None
    return getattr(stream, "cuda_stream", stream) or None


def _prec(p) -> int:
    return PREC[p] if isinstance(p, str) else int(p)


class Handle:
    """A libdwf handle (dwf_t).  Keeps the links tensor it was created with alive."""

    def __init__(self, dims, Ls, M5, mf, b, c, links, stream=None):
        lib = load()
        self._h = ctypes.c_void_p()
        self.dims = tuple(int(v) for v in dims)
        self.Ls, self.M5, self.mf, self.b, self.c = int(Ls), float(M5), float(mf), float(b), float(c)
        arr = (ctypes.c_int * 4)(*self.dims)
        _check(lib.dwf_create(ctypes.byref(self._h), arr, self.Ls, self.M5, self.mf, self.b,
                              self.c, _ptr(links), _stream_ptr(stream)))

    @property
    def ptr(self):
        return self._h

    def close(self):
        if self._h:
            load().dwf_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dwf_create(dims, Ls, M5, mf, b, c, links, stream=None) -> Handle:
    return Handle(dims, Ls, M5, mf, b, c, links, stream)


def dwf_update_links(h: Handle, links):
    _check(load().dwf_update_links(h.ptr, _ptr(links)))


def dwf_apply(h: Handle, op, inp, out, prec="f64"):
    op = OPS[op] if isinstance(op, str) else int(op)
    _check(load().dwf_apply(h.ptr, op, _ptr(inp), _ptr(out), _prec(prec)))
    return out


def dwf_cg(h: Handle, phi, x, tol, maxit, prec="f64", history: int = 0, raise_on_fail=True,
           curvature: bool = False):
    """history: record up to this many relative residual norms; curvature: also record
    <p_k, A p_k> / ||phi||^2 per iteration (the Lanczos coefficients of FP64 CG)."""
    st = Stats()
    buf = cbuf = None
    if history:
        buf = (ctypes.c_double * history)()
        st.history = buf
        st.history_capacity = history
        if curvature:
            cbuf = (ctypes.c_double * history)()
            st.curvature_history = cbuf
    s = load().dwf_cg(h.ptr, _ptr(phi), _ptr(x), float(tol), int(maxit), _prec(prec),
                      ctypes.byref(st))
    _check(s, () if raise_on_fail else (DWF_ERR_NOT_CONVERGED,))
    out = st.as_dict()
    out["status"] = s
    return out


def dwf_mspcg(h: Handle, block, inner_iters, inner, middle, phi, x, tol, maxit,
              local_op=LOCAL_DROP, flexible=False, history: int = 0, raise_on_fail=True):
    st = Stats()
    buf = None
    if history:
        buf = (ctypes.c_double * history)()
        st.history = buf
        st.history_capacity = history
    blk = (ctypes.c_int * 4)(*[int(v) for v in block])
    s = load().dwf_mspcg(h.ptr, blk, int(inner_iters), _prec(inner), _prec(middle),
                         int(local_op), int(bool(flexible)), _ptr(phi), _ptr(x), float(tol),
                         int(maxit), ctypes.byref(st))
    _check(s, () if raise_on_fail else (DWF_ERR_NOT_CONVERGED,))
    out = st.as_dict()
    out["status"] = s
    return out


def dwf_ms_solve(h: Handle, block, inner_iters, inner, colours, phi, x, tol, maxit,
                 local_op=LOCAL_EXACT, history: int = 0, raise_on_fail=True):
    """Stationary block iteration: colours 1 (multisplitting iteration), 2 or 16 (Schwarz)."""
    st = Stats()
    buf = None
    if history:
        buf = (ctypes.c_double * history)()
        st.history = buf
        st.history_capacity = history
    blk = (ctypes.c_int * 4)(*[int(v) for v in block])
    s = load().dwf_ms_solve(h.ptr, blk, int(inner_iters), _prec(inner), int(local_op),
                            int(colours), _ptr(phi), _ptr(x), float(tol), int(maxit),
                            ctypes.byref(st))
    _check(s, () if raise_on_fail else (DWF_ERR_NOT_CONVERGED,))
    out = st.as_dict()
    out["status"] = s
    return out


def dwf_force(h: Handle, phi, X, dSdU, tol=1e-12):
    _check(load().dwf_force(h.ptr, _ptr(phi), _ptr(X) if X is not None else None, _ptr(dSdU),
                            float(tol)))
    return dSdU


def dwf_action(h: Handle, phi, X=None, tol=1e-12) -> float:
    S = ctypes.c_double()
    _check(load().dwf_action(h.ptr, _ptr(phi), _ptr(X) if X is not None else None, float(tol),
                             ctypes.byref(S)))
    return S.value


def dwf_batch_solve(problems, tol, maxit, stream=None):
    """problems: list of dicts with dims, Ls, M5, mf, b, c, links, phi, x (tensors/arrays);
    solves every A_i x_i = phi_i to tol and returns the per-problem statistics."""
    n = len(problems)
    arr = (Problem * n)()
    for i, p in enumerate(problems):
        arr[i].dims = (ctypes.c_int * 4)(*p["dims"])
        arr[i].Ls = p["Ls"]
        arr[i].M5, arr[i].mf, arr[i].b, arr[i].c = p["M5"], p["mf"], p["b"], p["c"]
        arr[i].links = _ptr(p["links"])
        arr[i].phi = _ptr(p["phi"])
        arr[i].x = _ptr(p["x"])
    stats = (Stats * n)()
    s = load().dwf_batch_solve(n, arr, float(tol), int(maxit), stats, _stream_ptr(stream))
    _check(s)
    return [stats[i].as_dict() for i in range(n)]


def dwf_profile_enable(h: Handle, on: bool = True):
    _check(load().dwf_profile_enable(h.ptr, int(bool(on))))


def dwf_profile_read(h: Handle) -> list:
    """Per-kernel-class launches, event-timed milliseconds, algorithmic bytes and flops since
    the last read (the counters are reset)."""
    cap = 64
    arr = (KernelProfile * cap)()
    n = ctypes.c_int()
    _check(load().dwf_profile_read(h.ptr, arr, cap, ctypes.byref(n)))
    return [dict(name=arr[i].name.decode(), launches=arr[i].launches, ms=arr[i].ms_total,
                 bytes=arr[i].bytes_total, flops=arr[i].flops_total) for i in range(n.value)]


def dwf_mdagm_noalloc(dims, Ls, M5, mf, b, c, links, inp, out, prec="f64", stream=None):
    """A = Mpc^dag Mpc for callers that cannot allocate device memory: device buffers only,
    all scratch in the library's static device array; queued on the stream, not synchronised."""
    arr = (ctypes.c_int * 4)(*[int(v) for v in dims])
    _check(load().dwf_mdagm_noalloc(arr, int(Ls), float(M5), float(mf), float(b), float(c),
                                    _ptr(links), _ptr(inp), _ptr(out), _prec(prec),
                                    _stream_ptr(stream)))
    return out


def dwf_set_option(h: Handle, option: int, value: float):
    """Per-handle option: OPT_WAIT_LIMIT_US (bounded device waits) or OPT_TEST_WAIT_PROBE."""
    _check(load().dwf_set_option(h.ptr, int(option), float(value)))


def dwf_measure_peak(which: str = "f64", stream=None) -> float:
    """Measured FMA peak of the current device in TFLOP/s ("f64": DFMA, "f32": FFMA)."""
    t = ctypes.c_double()
    _check(load().dwf_measure_peak({"f64": 0, "f32": 1}[which], _stream_ptr(stream),
                                   ctypes.byref(t)))
    return t.value
