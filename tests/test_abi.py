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


def test_more_validation_without_gpu(lib):
    """Batched create, solve, stats and the allocation-free product reject bad
    arguments before any CUDA call (include/bse.h states each rule)."""
    from paper_2504_10096_gb300 import bse
    h = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)
    ns = (ctypes.c_int64 * 2)(100, 200)
    ptrs = (ctypes.c_void_p * 2)(16, 16)
    nulls = (ctypes.c_void_p * 2)(16, None)

    def create_batched(count, n, a, b, form=1, dtype=1, where=1, out=True):
        return lib.bse_create_batched(count, n, a, b, form, dtype, where, None,
                                      ctypes.byref(h) if out else None)
    assert create_batched(2, ns, ptrs, ptrs, out=False) == bse.BSE_EINVAL
    assert create_batched(0, ns, ptrs, ptrs) == bse.BSE_EINVAL
    assert create_batched(2, None, ptrs, ptrs) == bse.BSE_EINVAL
    assert create_batched(2, ns, None, ptrs) == bse.BSE_EINVAL
    assert create_batched(2, ns, ptrs, None) == bse.BSE_EINVAL          # PH without B
    assert create_batched(2, ns, ptrs, nulls) == bse.BSE_EINVAL         # PH, one B missing
    assert create_batched(2, ns, nulls, ptrs) == bse.BSE_EINVAL         # one A missing
    assert create_batched(2, (ctypes.c_int64 * 2)(100, 0), ptrs, ptrs) == bse.BSE_EINVAL
    assert create_batched(2, (ctypes.c_int64 * 2)(100, 1 << 31), ptrs, ptrs) == bse.BSE_EINVAL
    assert create_batched(2, ns, ptrs, ptrs, form=3) == bse.BSE_EINVAL
    assert create_batched(2, ns, ptrs, ptrs, dtype=4) == bse.BSE_EINVAL
    assert create_batched(2, ns, ptrs, ptrs, where=2) == bse.BSE_EINVAL
    assert h.value is None                                              # *out cleared on failure

    ev = (ctypes.c_double * 4)()
    n = ctypes.c_int(0)
    assert lib.bse_solve(None, 4, 1e-10, 0, ev, None, ctypes.byref(n)) == bse.BSE_EINVAL
    assert lib.bse_solve_ex(None, 4, 1e-10, 0, None, ev, None, ctypes.byref(n)) == bse.BSE_EINVAL
    assert lib.bse_solve_batched(None, 4, 1e-10, 0, None, ev, None, None) == bse.BSE_EINVAL
    st = bse.bse_stats()
    assert lib.bse_get_stats(None, ctypes.byref(st)) == bse.BSE_EINVAL

    def noalloc(N, A, B, dtype, op, x, y):
        return lib.bse_apply_noalloc(N, A, B, dtype, op, x, y, None)
    assert noalloc(0, dummy, dummy, 1, 1, dummy, dummy) == bse.BSE_EINVAL
    assert noalloc(bse.BSE_NOALLOC_MAX_N + 1, dummy, dummy, 1, 1, dummy, dummy) == bse.BSE_EINVAL
    assert noalloc(10, None, dummy, 1, 1, dummy, dummy) == bse.BSE_EINVAL
    assert noalloc(10, dummy, None, 1, bse.BSE_OP_MPLUS, dummy, dummy) == bse.BSE_EINVAL
    assert noalloc(10, dummy, None, 1, bse.BSE_OP_MMINUS, dummy, dummy) == bse.BSE_EINVAL
    assert noalloc(10, dummy, dummy, 1, bse.BSE_OP_H, dummy, dummy) == bse.BSE_EINVAL
    assert noalloc(10, dummy, dummy, bse.BSE_C128_DF, 1, dummy, dummy) == bse.BSE_EINVAL
    assert noalloc(10, dummy, dummy, 1, 1, None, dummy) == bse.BSE_EINVAL
    assert noalloc(10, dummy, dummy, 1, 1, dummy, None) == bse.BSE_EINVAL


def test_newer_entry_points_validate_without_gpu(lib):
    """The dense solve, the mixed product, the residual query and the FP64 peak
    measurement reject bad arguments before any CUDA call."""
    from paper_2504_10096_gb300 import bse
    dummy = ctypes.c_void_p(16)
    ev = (ctypes.c_double * 4)()
    n = ctypes.c_int(0)
    assert lib.bse_solve_dense(None, 4, 1e-10, ev, None, ctypes.byref(n)) == bse.BSE_EINVAL
    assert lib.bse_apply_mixed(None, bse.BSE_OP_MPLUS, 0.0, dummy, dummy) == bse.BSE_EINVAL
    assert lib.bse_get_residuals(None, 0, ev, 4) == bse.BSE_EINVAL
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    assert lib.bse_measure_fp64_peak(0, ctypes.byref(tf), ctypes.byref(ms)) == bse.BSE_EINVAL
    assert lib.bse_measure_fp64_peak(1 << 25, ctypes.byref(tf), ctypes.byref(ms)) == bse.BSE_EINVAL
    assert lib.bse_measure_fp64_peak(100, None, None) == bse.BSE_EINVAL


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of bse_solve_opts and bse_stats have the C layout
    (offset of every field and the size), checked against gcc on the header."""
    import shutil
    import subprocess
    from paper_2504_10096_gb300 import bse
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bse.h"', "int main(void) {"]
    for cls in (bse.bse_solve_opts, bse.bse_stats):
        name = cls.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            name, field, val = line.split()
            got[(name, field)] = int(val)
    for cls in (bse.bse_solve_opts, bse.bse_stats):
        name = cls.__name__
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)

