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


@pytest.mark.parametrize("n", [129, 515])
def test_mixed_product_exact_and_coarse_tiles(n):
    """The mixed path's product (bse_apply_mixed, complex128 vectors) on a
    complex64 handle.  Every tile exact (tile_tau < 0, double-FP32): within a
    few 2^-48 of |M||x| per entry of the oracle's M+/M- x.  Every tile coarse
    (tile_tau = 1): U = A + sB, V = A - sB rounded to FP32 on purpose, so the
    reference is the real form of Eq. 5 applied with those rounded blocks in
    FP64; the fixed-point-grid accumulation must match it to 2^-30 of the
    largest |U||x| row sum (plain FP32 accumulation would be near 2^-22)."""
    from paper_2504_10096_gb300 import bse
    A, B = problem(n, "c64", seed=n + 21)
    s = bse.Solver(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), mixed=True)
    x = rand_block(n, 1, "c128", seed=9)
    xt = torch.from_numpy(x[:, 0]).cuda()
    A64, B64 = A.astype(np.complex128), B.astype(np.complex128)
    for op, sgn, fn in ((bse.BSE_OP_MPLUS, 1.0, O.apply_mplus), (bse.BSE_OP_MMINUS, -1.0, O.apply_mminus)):
        y = torch.empty_like(xt)
        assert bse.bse_apply_mixed(s.h, op, -1.0, xt.data_ptr(), y.data_ptr()) == bse.BSE_OK
        assert s.stats()["tiles_coarse"] == 0
        ref = fn(A64, B64, x)
        assert_elementwise(y.cpu().numpy()[:, None], ref, product_bound(A, B, x, "mplus"), 2.0 ** -48, 64,
                           f"mixed exact, sign {sgn}")
        assert bse.bse_apply_mixed(s.h, op, 1.0, xt.data_ptr(), y.data_ptr()) == bse.BSE_OK
        assert s.stats()["tiles_fine"] == 0 and s.stats()["tiles_coarse"] > 0
        f32 = np.float32
        ure = (A.real.astype(f32) + f32(sgn) * B.real.astype(f32)).astype(np.float64)
        uim = (A.imag.astype(f32) + f32(sgn) * B.imag.astype(f32)).astype(np.float64)
        vre = (A.real.astype(f32) - f32(sgn) * B.real.astype(f32)).astype(np.float64)
        vim = (A.imag.astype(f32) - f32(sgn) * B.imag.astype(f32)).astype(np.float64)
        xr, xi = x[:, 0].real, x[:, 0].imag
        emu = (ure @ xr - vim @ xi) + 1j * (uim @ xr + vre @ xi)
        scale = np.max((np.abs(ure) + np.abs(vim) + np.abs(uim) + np.abs(vre)) @ np.abs(x[:, 0]))
        err = np.max(np.abs(y.cpu().numpy() - emu))
        assert err <= 2.0 ** -30 * scale, (sgn, err / scale)
    s.close()
