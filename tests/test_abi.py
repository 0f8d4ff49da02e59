"""The C ABI library builds for sm_103a, loads without a GPU, and exports every function that
include/dwf.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dwf.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dwf_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dwf_create", "dwf_apply", "dwf_cg", "dwf_mspcg", "dwf_force",
                     "dwf_destroy", "dwf_last_error"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1804_08593_gb300 import build, dwf
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(dwf.EXPORTS) == set(declared_functions())
    loaded = dwf.load()
    assert loaded.dwf_version().decode().startswith("dwf-gb300")
    assert isinstance(dwf.dwf_last_error(), str)


def test_binding_rejects_wrong_dtypes():
    import numpy as np
    from paper_1804_08593_gb300 import dwf
    with pytest.raises(ValueError):
        dwf._ptr(np.zeros(4, dtype=np.complex64))
    with pytest.raises(ValueError):
        dwf._ptr(np.zeros((4, 4), dtype=np.complex128)[:, ::2])


def test_argument_errors_are_status_codes_before_any_device_call():
    """Invalid arguments come back as DWF_ERR_ARG with a message, checked on the host before
    the library touches the device (so this runs without a GPU)."""
    from paper_1804_08593_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.dwf_last_error.restype = ctypes.c_char_p
    ERR_ARG = 1
    D = ctypes.c_double
    create = lib.dwf_create
    create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                       D, D, D, D, ctypes.c_void_p, ctypes.c_void_p]
    h = ctypes.c_void_p(1)
    links = ctypes.c_void_p(0x1000)   # never dereferenced: every call below fails its checks first

    def dims(*d):
        return (ctypes.c_int * 4)(*d)

    def last():
        return lib.dwf_last_error().decode()

    assert create(ctypes.byref(h), dims(4, 4, 4, 4), 8, 1.8, 0.1, 1.5, 0.5, None, None) == ERR_ARG
    assert "null" in last()
    assert create(ctypes.byref(h), dims(4, 3, 4, 4), 8, 1.8, 0.1, 1.5, 0.5, links, None) == ERR_ARG
    assert "even" in last() and h.value is None          # the handle is cleared on failure
    assert create(ctypes.byref(h), dims(4, 4, 0, 4), 8, 1.8, 0.1, 1.5, 0.5, links, None) == ERR_ARG
    assert create(ctypes.byref(h), dims(4, 4, 4, 4), 5, 1.8, 0.1, 1.5, 0.5, links, None) == ERR_ARG
    assert "Ls must be one of" in last()

    lib.dwf_apply.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_int]
    assert lib.dwf_apply(None, 1, links, links, 0) == ERR_ARG and "null" in last()

    lib.dwf_batch_solve.argtypes = [ctypes.c_int, ctypes.c_void_p, D, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_void_p]
    assert lib.dwf_batch_solve(0, None, 1e-10, 100, None, None) == ERR_ARG
    assert "no problems" in last()

    na = lib.dwf_mdagm_noalloc
    na.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_int, D, D, D, D, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    buf = ctypes.c_void_p(0x2000)
    assert na(dims(4, 4, 4, 4), 8, 1.8, 0.1, 1.5, 0.5, links, buf, buf, 1, None) == ERR_ARG
    assert "alias" in last()
    assert na(dims(4, 4, 4, 4), 8, 1.8, 0.1, 1.5, 0.5, links, links, buf, 7, None) == ERR_ARG
    assert "precision" in last()
    assert na(dims(4, 4, 4, 4), 7, 1.8, 0.1, 1.5, 0.5, links, links, buf, 1, None) == ERR_ARG
    assert na(dims(2, 2, 2, 5), 8, 1.8, 0.1, 1.5, 0.5, links, links, buf, 1, None) == ERR_ARG

    lib.dwf_destroy.argtypes = [ctypes.c_void_p]
    lib.dwf_destroy(None)                                   # a null handle is ignored
