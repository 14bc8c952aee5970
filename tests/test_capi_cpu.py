"""CPU checks of the boundary: the library builds for sm_103a, loads without a
GPU, exports every entry point the header declares, and rejects invalid
arguments before touching the device."""
import ctypes
import os
import re

import pytest

from paper_0706_0747_gb300 import build as B
from paper_0706_0747_gb300 import mra

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "mra_gb300.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB):
        B.build()
    return mra.lib()


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*|unsigned long long)\s+(mra_\w+)\s*\(", txt, re.M)))


def test_header_declares_entry_points():
    names = declared()
    for n in ["mra_build_tree", "mra_compress", "mra_make_operator", "mra_apply_ns", "mra_reconstruct",
              "mra_free_tree", "mra_free_op"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_covers_header():
    assert sorted(mra.symbols_declared()) == declared()


def test_invalid_arguments_rejected_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.mra_make_operator(0.0, 2.0, 1e-6, 8, 7, None, None, ctypes.byref(h)) == mra.EINVAL
    assert "alpha" in mra.last_error()
    assert lib.mra_make_operator(0.0, 1.0, 0.0, 8, 7, None, None, ctypes.byref(h)) == mra.EINVAL
    assert lib.mra_make_operator(0.0, 1.0, 1e-6, 0, 7, None, None, ctypes.byref(h)) == mra.EINVAL
    assert lib.mra_make_operator(-1.0, 1.0, 1e-6, 8, 7, None, None, ctypes.byref(h)) == mra.EINVAL
    assert lib.mra_make_operator(0.0, 1.0, 1e-6, 8, 99, None, None, ctypes.byref(h)) == mra.EINVAL
    assert h.value is None
    d = mra.Density(0, None, None, None, None)
    assert lib.mra_build_tree(ctypes.byref(d), 8, 1e-6, 7, -1, 0, None, None, ctypes.byref(h)) == mra.EINVAL
    assert lib.mra_free_tree(None) == mra.OK and lib.mra_free_op(None) == mra.OK


def test_version(lib):
    assert "sm_103a" in mra.version()
