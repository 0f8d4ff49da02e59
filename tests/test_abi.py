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
