"""bse_apply_noalloc: the product for callers that cannot let the library
allocate device memory (a pool-owned device, or a loop where cudaMalloc's
possible device synchronisation is not acceptable).  Checked through the C ABI
against the handle-based bse_apply on two calls in a row (the shared scratch
array keeps the previous call's contents), with the tolerances of the other
product tests, and element by element against the oracle's operators with
the bound of tests/test_gpu_product.py.  Kept in its own file so that a run
stopping at the first failure has already run every other test."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import UNIT, assert_elementwise, problem, product_bound, rand_block, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"c128": 1e-13, "c64": 3e-6}


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [1000, 4096])
def test_noalloc_matches_bse_apply(dtype, n):
    from paper_2504_10096_gb300 import bse
    A, B = problem(n, dtype, seed=n + 11, n_g=64)
    At = torch.from_numpy(A).cuda()
    Bt = torch.from_numpy(B).cuda()
    s = bse.Solver(At, Bt)
    code = bse.BSE_C128 if dtype == "c128" else bse.BSE_C64
    stream = torch.cuda.current_stream()
    oracle_ops = {bse.BSE_OP_A: (O.apply_a, "a"), bse.BSE_OP_MPLUS: (O.apply_mplus, "mplus"),
                  bse.BSE_OP_MMINUS: (O.apply_mminus, "mminus")}
    for call, seed in enumerate((1, 2)):            # two calls in a row, different inputs
        xh = rand_block(n, 1, dtype, seed=seed)
        x = torch.from_numpy(xh[:, 0]).cuda()
        for op in (bse.BSE_OP_A, bse.BSE_OP_MPLUS, bse.BSE_OP_MMINUS):
            ref = s.apply(op, x).cpu().numpy()
            y = torch.empty_like(x)
            rc = bse.bse_apply_noalloc(n, At.data_ptr(), Bt.data_ptr(), code, op, x.data_ptr(),
                                       y.data_ptr(), stream.cuda_stream)
            assert rc == bse.BSE_OK
            torch.cuda.synchronize()
            yh = y.cpu().numpy()
            assert rel(yh, ref) < TOL[dtype], (call, op)
            fn, name = oracle_ops[op]
            oref = fn(A, xh) if op == bse.BSE_OP_A else fn(A, B, xh)
            assert_elementwise(yh[:, None], oref, product_bound(A, B, xh, name), UNIT[dtype], 64,
                               f"noalloc op {name}, call {call}")
    s.close()


def test_noalloc_rejects_mixed_dtype():
    """BSE_C64_MIXED names a handle layout (FP64 basis) that a handle-free call has
    no use for: the entry point takes BSE_C64 or BSE_C128 only."""
    from paper_2504_10096_gb300 import bse
    dummy = torch.zeros(4, dtype=torch.complex64, device="cuda")
    rc = bse.bse_apply_noalloc(2, dummy.data_ptr(), dummy.data_ptr(), bse.BSE_C64_MIXED, bse.BSE_OP_MPLUS,
                               dummy.data_ptr(), dummy.data_ptr(), 0)
    assert rc == bse.BSE_EINVAL


def test_noalloc_rejects_oversize():
    from paper_2504_10096_gb300 import bse
    n = bse.BSE_NOALLOC_MAX_N + 1
    dummy = torch.zeros(4, dtype=torch.complex128, device="cuda")
    rc = bse.bse_apply_noalloc(n, dummy.data_ptr(), dummy.data_ptr(), bse.BSE_C128, bse.BSE_OP_MPLUS,
                               dummy.data_ptr(), dummy.data_ptr(), 0)
    assert rc == bse.BSE_EINVAL
    assert "invalid" in bse.bse_strerror(rc)
