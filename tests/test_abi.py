"""CPU checks of the C ABI: the library builds, loads, exports every function
include/bse.h declares, and its argument validation answers without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bse.h")).read()
    return sorted(set(re.findall(r"\b(bse_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_10096_gb300 import bse, build
    if not os.path.exists(bse.LIB_PATH):
        build.build()
    return bse.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "bse_create" in names and "bse_solve" in names and "bse_backward" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_abi():
    from paper_2504_10096_gb300 import bse
    assert set(_declared()) <= set(bse.EXPORTED)


def test_strerror_and_validation_without_gpu(lib):
    from paper_2504_10096_gb300 import bse
    for code in range(9):
        assert len(bse.bse_strerror(code)) > 3
    h = ctypes.c_void_p()
    # invalid sizes / enums are rejected before any CUDA call
    assert lib.bse_create(0, None, None, 0, 1, 1, None, ctypes.byref(h)) == bse.BSE_EINVAL
    assert lib.bse_create(10, None, None, 0, 1, 1, None, ctypes.byref(h)) == bse.BSE_EINVAL
    dummy = ctypes.c_void_p(16)
    assert lib.bse_create(10, dummy, None, 1, 1, 1, None, ctypes.byref(h)) == bse.BSE_EINVAL  # PH without B
    assert lib.bse_create(10, dummy, dummy, 5, 1, 1, None, ctypes.byref(h)) == bse.BSE_EINVAL
    assert lib.bse_create(10, dummy, dummy, 1, 9, 1, None, ctypes.byref(h)) == bse.BSE_EINVAL
    assert lib.bse_create(10, dummy, dummy, 1, 1, 7, None, ctypes.byref(h)) == bse.BSE_EINVAL
    assert lib.bse_destroy(None) == bse.BSE_EINVAL
    assert lib.bse_apply(None, 0, 1, dummy, dummy) == bse.BSE_EINVAL
    assert lib.bse_backward(None, None, 0, None, None) == bse.BSE_EINVAL
    assert lib.bse_backward_ex(None, None, 0, None, None, 0) == bse.BSE_EINVAL
    w = (ctypes.c_double * 4)(1.0, 2.0, 3.0, 4.0)
    out = (ctypes.c_double * 4)()
    assert lib.bse_haydock(None, dummy, 1, 10, -1, 4, w, 0.1, out, None, None, None) == bse.BSE_EINVAL
    e = ctypes.c_int(0)
    assert lib.bse_selftest_bounded_wait(2, ctypes.byref(e)) == bse.BSE_EINVAL
    assert lib.bse_selftest_bounded_wait(0, None) == bse.BSE_EINVAL


def test_missing_library_fails_loudly(tmp_path):
    from paper_2504_10096_gb300 import bse
    saved = bse._LIB
    bse._LIB = None
    try:
        with pytest.raises(RuntimeError):
            bse.load_library(str(tmp_path / "nope.so"))
    finally:
        bse._LIB = saved
