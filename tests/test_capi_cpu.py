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
    return sorted(set(re.findall(r"^\s*(?:int|const char\*|unsigned long long|size_t)\s+(mra_\w+)\s*\(", txt, re.M)))


def test_header_declares_entry_points():
    names = declared()
    for n in ["mra_build_tree", "mra_compress", "mra_make_operator", "mra_apply_ns", "mra_reconstruct",
              "mra_free", "mra_free_tree", "mra_free_op"]:
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


def test_compress_modes_and_cache_without_gpu(lib):
    # the compress modes are ABI constants; a bad handle is refused before any mode check
    assert (mra.COMPRESS_NORMS, mra.COMPRESS_STORE_D, mra.COMPRESS_SCALING) == (0, 1, 2)
    for mode in (0, 1, 2, 3):
        assert lib.mra_compress(None, mode, None) == mra.EINVAL
    assert "tree handle" in mra.last_error()
    # releasing empties the reuse cache: a second release finds nothing
    assert mra.release_cached() >= 0
    assert mra.release_cached() == 0


def test_batched_and_schedule_entries_reject_invalid_arguments(lib):
    """Argument checks of the batched, network and no-alloc entries that run
    before any device work (so they need no GPU)."""
    h = ctypes.c_void_p()
    # a plan needs an operator and at least one tree
    assert lib.mra_plan_create(None, None, 0, None, None, ctypes.byref(h)) == mra.EINVAL
    assert h.value is None
    for fn, args in [("mra_plan_execute", (None, None)), ("mra_plan_autotune", (None, 1, None)),
                     ("mra_plan_set_variant", (None, 8, 2, 0)), ("mra_plan_get_info", (None, None, None)),
                     ("mra_plan_tree_stats", (None, 0, None, None)), ("mra_screen_data", (None, None, None, None, None)),
                     ("mra_mlp_forward", (None, None, 0, None, None)), ("mra_mlp_num_params", (None, None)),
                     ("mra_apply_ns_noalloc", (None, None, 0, None, None, None))]:
        assert getattr(lib, fn)(*args) == mra.EINVAL, fn
    p = ctypes.c_void_p()
    assert lib.mra_plan_output(None, 0, None, ctypes.byref(p)) == mra.EINVAL and p.value is None
    # network shapes outside [1, 1024]
    assert lib.mra_mlp_create(0, 12, None, 0, None, None, ctypes.byref(h)) == mra.EINVAL
    assert lib.mra_mlp_create(16, 2000, None, 0, None, None, ctypes.byref(h)) == mra.EINVAL
    assert h.value is None
    assert lib.mra_free_plan(None) == mra.OK and lib.mra_mlp_free(None) == mra.OK


def test_mra_free_dispatch_rejects_non_handles(lib):
    """mra_free(NULL) is a no-op; memory that does not start with a handle tag
    is refused with MRA_EINVAL (no device call is made)."""
    assert lib.mra_free(None) == mra.OK
    junk = ctypes.create_string_buffer(b"\x00" * 64)
    assert lib.mra_free(ctypes.cast(junk, ctypes.c_void_p)) == mra.EINVAL
    assert "not a live handle" in mra.last_error()
