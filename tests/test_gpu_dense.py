"""GPU parity of the dense structure-preserving diagonalisation (bse_solve_dense:
M_r of Eq. 5, Cholesky, W = L^T J L, skew-tridiagonal reduction, bisection and
inverse iteration, back-transformation) against the dense FP64 oracle (zgeev of
the full 2N matrix), with sizes that span one 64-column panel, several, and a
ragged tail, and a share of the spectrum above the iterative regime."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import omega_metric_apply, problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _solver(A, B, **kw):
    from paper_2504_10096_gb300 import bse
    return bse.Solver(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), **kw)


@pytest.mark.parametrize("n,nev", [(1, 1), (5, 5), (37, 10), (64, 20), (129, 40), (300, 120)])
def test_dense_fp64_against_zgeev(n, nev):
    A, B = problem(n, "c128", seed=200 + n)
    s = _solver(A, B)
    vals, vecs, nconv = s.solve_dense(nev, tol=1e-10)
    om, Xo, Yo = O.ph_lowest(A, B, nev)
    assert nconv == nev
    np.testing.assert_allclose(vals, om, rtol=1e-10, atol=0)
    assert s.residuals().max() <= 1e-10
    Z = vecs.cpu().numpy()
    jn = np.real(np.einsum("ij,ij->j", Z.conj(), omega_metric_apply(Z)))
    np.testing.assert_allclose(jn, 1.0, atol=1e-10)
    gaps = np.diff(om)
    simple = np.ones(nev, bool)
    if nev > 1:
        simple[1:] &= gaps > 1e-6
        simple[:-1] &= gaps > 1e-6
    ov = np.abs(np.einsum("ij,ij->j", Z.conj(), omega_metric_apply(np.vstack([Xo, Yo]))))
    np.testing.assert_allclose(ov[simple], 1.0, atol=1e-7)
    s.close()


def test_dense_complex64_storage_and_config4_recipe():
    """complex64 A and B (promoted to FP64 on the device) from the config-4 recipe
    (energies in [1, 12] eV, N_G = 2000) at N = 800, 20 % of the positive spectrum:
    eigenvalues against the oracle's dense reduction of the same values."""
    from synthetic import make_problem, reduced_spec
    spec = reduced_spec(4, 800)
    p = make_problem(spec)
    A, B = p["A"], p["B"]
    nev = 160
    s = _solver(A, B)
    vals, _, nconv = s.solve_dense(nev, tol=1e-10, vectors=False)
    ref = O.ph_lowest_shao(A, B, nev)
    assert nconv == nev
    np.testing.assert_allclose(vals, ref, rtol=1e-10, atol=0)
    s.close()


def test_dense_matches_iterative():
    """The dense and the iterative solver agree on the same handle (FP64)."""
    A, B = problem(400, "c128", seed=211)
    s = _solver(A, B)
    v1, _, _ = s.solve(12, tol=1e-12)
    v2, _, _ = s.solve_dense(12, tol=1e-10)
    np.testing.assert_allclose(v2, v1, rtol=1e-11, atol=0)
    s.close()


def test_dense_not_positive_definite_and_invalid():
    from paper_2504_10096_gb300 import bse
    n = 70
    s = _solver(np.eye(n, dtype=np.complex128), 2.0 * np.eye(n, dtype=np.complex128))
    rc, _, _ = bse.bse_solve_dense(s.h, 4, 1e-10)
    assert rc == bse.BSE_ENOTPD
    s.close()
    A, _ = problem(50, "c128", form="tda", seed=3)
    t = bse.Solver(torch.from_numpy(A).cuda())
    rc, _, _ = bse.bse_solve_dense(t.h, 4, 1e-10)
    assert rc == bse.BSE_EINVAL
    t.close()
