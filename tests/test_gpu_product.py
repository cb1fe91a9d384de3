"""GPU parity of the structured products (bse_apply) against the oracle's
plain definitions: Y = A X, M+ X = A X + B conj(X), M- X = A X - B conj(X),
and Y = H X with H of Eq. 1, for single vectors (the streaming tile kernel
of the Lanczos steps) and blocks (the row-block kernel).  Sizes span one
tile, exact multiples of the 128 tile edge and ragged tails.

Every entry is checked against the oracle's value on its own:
|Y - Y_oracle|_i <= c u (|M| |X|)_i, with u the unit roundoff of the storage
precision and c a small constant covering the accumulation depth (at most a
few tens of roundings per entry) and the conversion of the vector."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import UNIT, assert_elementwise, problem, product_bound, rand_block, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _solver(A, B):
    from paper_2504_10096_gb300 import bse
    return bse.Solver(torch.from_numpy(A).cuda(), None if B is None else torch.from_numpy(B).cuda())


TOL = {"c128": 1e-13, "c64": 3e-6}
C_ELEM = 64        # roundings per entry allowed by the element-wise bound


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 37, 128, 129, 300, 515])
@pytest.mark.parametrize("k", [1, 3])
def test_apply_ph_ops(dtype, n, k):
    from paper_2504_10096_gb300 import bse
    A, B = problem(n, dtype, seed=n)
    s = _solver(A, B)
    X = rand_block(n, k, dtype, seed=1)
    Xt = torch.from_numpy(X).cuda()
    refs = {bse.BSE_OP_A: (O.apply_a(A, X), "a"), bse.BSE_OP_MPLUS: (O.apply_mplus(A, B, X), "mplus"),
            bse.BSE_OP_MMINUS: (O.apply_mminus(A, B, X), "mminus")}
    for op, (ref, name) in refs.items():
        Y = s.apply(op, Xt).cpu().numpy()
        assert rel(Y, ref) < TOL[dtype], (op, rel(Y, ref))
        assert_elementwise(Y, ref, product_bound(A, B, X, name), UNIT[dtype], C_ELEM, f"op {name}")
    Z = rand_block(2 * n, k, dtype, seed=2)
    Y = s.apply(bse.BSE_OP_H, torch.from_numpy(Z).cuda()).cpu().numpy()
    ref = O.apply_bse(A, B, Z)
    assert rel(Y, ref) < TOL[dtype]
    assert_elementwise(Y, ref, product_bound(A, B, Z, "h"), UNIT[dtype], C_ELEM, "op H")
    s.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_lower_triangle_is_ignored_and_host_input(dtype):
    """Only the upper triangle is read; host (numpy) input gives the same bytes."""
    from paper_2504_10096_gb300 import bse
    n = 261
    A, B = problem(n, dtype, seed=5)
    junk = A.copy()
    junk[np.tril_indices(n, -1)] = 7.0 + 3.0j
    junkb = B.copy()
    junkb[np.tril_indices(n, -1)] = -2.0 + 1.0j
    X = rand_block(n, 1, dtype, seed=3)
    s1 = bse.Solver(torch.from_numpy(junk).cuda(), torch.from_numpy(junkb).cuda())
    s2 = bse.Solver(A, B)          # numpy -> host copy path
    for op in (bse.BSE_OP_MPLUS, bse.BSE_OP_MMINUS):
        y1 = s1.apply(op, torch.from_numpy(X).cuda()).cpu().numpy()
        y2 = s2.apply(op, torch.from_numpy(X).cuda()).cpu().numpy()
        ref = O.apply_mplus(A, B, X) if op == bse.BSE_OP_MPLUS else O.apply_mminus(A, B, X)
        assert rel(y1, ref) < TOL[dtype] and rel(y2, ref) < TOL[dtype]
        bnd = product_bound(A, B, X, "mplus")
        assert_elementwise(y1, ref, bnd, UNIT[dtype], C_ELEM, "lower triangle ignored")
        assert_elementwise(y2, ref, bnd, UNIT[dtype], C_ELEM, "host input")
    s1.close()
    s2.close()


def test_tda_handle_apply():
    from paper_2504_10096_gb300 import bse
    n = 333
    A, _ = problem(n, "c128", form="tda", seed=9)
    s = _solver(A, None)
    X = rand_block(n, 5, "c128", seed=4)
    Y = s.apply(bse.BSE_OP_A, torch.from_numpy(X).cuda()).cpu().numpy()
    assert rel(Y, A @ X) < 1e-13
    assert_elementwise(Y, O.apply_a(A, X), product_bound(A, None, X, "a"), UNIT["c128"], C_ELEM, "TDA A X")
    with pytest.raises(bse.BSEError):
        s.apply(bse.BSE_OP_MPLUS, torch.from_numpy(X).cuda())
    s.close()


@pytest.mark.parametrize("n", [37, 129, 515])
def test_apply_df64_products(n):
    """complex128 handle with double-FP32 products (BSE_C128_DF): every op
    against the FP64 oracle; the per-term error is 2^-48, far below FP32."""
    from paper_2504_10096_gb300 import bse
    A, B = problem(n, "c128", seed=n + 3)
    s = bse.Solver(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), df=True)
    X = rand_block(n, 1, "c128", seed=5)
    Xt = torch.from_numpy(X).cuda()
    for op, ref, name in ((bse.BSE_OP_A, O.apply_a(A, X), "a"), (bse.BSE_OP_MPLUS, O.apply_mplus(A, B, X), "mplus"),
                          (bse.BSE_OP_MMINUS, O.apply_mminus(A, B, X), "mminus")):
        Y = s.apply(op, Xt).cpu().numpy()
        assert rel(Y, ref) < 1e-12, (op, rel(Y, ref))
        # double-FP32 terms carry 2^-48 relative error (the dropped lo x lo product)
        assert_elementwise(Y, ref, product_bound(A, B, X, name), 2.0 ** -48, C_ELEM, f"df op {name}")
    s.close()
