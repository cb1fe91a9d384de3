"""Edge cases of the iterative solver at the smallest sizes, against the dense oracle.

* N = 1 (closed forms: lambda = a for TDA, omega = sqrt(a^2 - |b|^2) for PH, Sec. 1);
* the subspace is the whole space (ncv capped at N, both forms): one cycle
  reaches an invariant subspace and must lock everything;
* pseudo-Hermitian with the subspace close to or equal to N (the folded
  operator's N-dimensional Krylov space): the projection onto the twins' space
  keeps the second copy of every omega^2 out, so the pairs reach tol;
* a caller-given ncv equal to nev (raised to nev + 1 so that every cycle adds a
  new Lanczos vector);
* a batch whose smallest problem caps ncv at nev while a larger one needs
  more: rejected (no cycle could add a vector to the larger problem)."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _solver(A, B=None):
    from paper_2504_10096_gb300 import bse
    return bse.Solver(torch.from_numpy(A).cuda(), None if B is None else torch.from_numpy(B).cuda())


def test_n1_tda_and_ph_closed_forms():
    a, b = 2.5, 0.7 * np.exp(0.3j)
    A = np.array([[a]], dtype=np.complex128)
    B = np.array([[b]], dtype=np.complex128)
    s = _solver(A)
    vals, vecs, nconv = s.solve(1, tol=1e-12)
    assert nconv == 1
    np.testing.assert_allclose(vals, [a], rtol=1e-14)
    assert abs(abs(vecs.cpu().numpy()[0, 0]) - 1.0) < 1e-14
    s.close()
    s = _solver(A, B)
    vals, vecs, nconv = s.solve(1, tol=1e-12)
    assert nconv == 1
    w = np.sqrt(a * a - abs(b) ** 2)
    np.testing.assert_allclose(vals, [w], rtol=1e-13)
    z = vecs.cpu().numpy()[:, 0]
    assert abs(abs(z[0]) ** 2 - abs(z[1]) ** 2 - 1.0) < 1e-12        # Omega-normalised
    assert abs((a - w) * z[0] + b * z[1]) < 1e-12 * abs(z[0])         # first row of (H - w) z = 0
    s.close()


def _check_pairs(form, A, B, n, nev, vals, vecs, nconv):
    ref = O.ph_lowest(A, B, nev)[0] if form == "ph" else O.tda_lowest(A, nev)[0]
    assert nconv == nev
    np.testing.assert_allclose(vals, ref, rtol=1e-11, atol=0)
    Z = vecs.cpu().numpy()
    res = O.relative_residuals_ph(A, B, vals, Z[:n], Z[n:]) if form == "ph" \
        else O.relative_residuals_tda(A, vals, Z)
    assert res.max() < 1e-11


@pytest.mark.parametrize("form,n,nev", [("tda", 40, 40), ("tda", 40, 10), ("tda", 2, 2), ("ph", 2, 2),
                                        ("ph", 40, 40), ("ph", 40, 39), ("ph", 40, 10)])
def test_subspace_is_the_whole_space(form, n, nev):
    """ncv is capped at N: the first cycle reaches an invariant subspace."""
    A, B = problem(n, "c128", form=form, seed=100 + n + nev)
    s = _solver(A, B if form == "ph" else None)
    vals, vecs, nconv = s.solve(nev, tol=1e-12)
    _check_pairs(form, A, B, n, nev, vals, vecs, nconv)
    assert s.residuals().max() <= 1e-12
    s.close()


@pytest.mark.parametrize("nev,ncv", [(10, 39), (38, 39), (10, 40), (39, 40)])
def test_ph_subspace_close_to_n(nev, ncv):
    """Pseudo-Hermitian N = 40 with ncv = N - 1 or N: every counted pair has an
    FP64 residual <= tol and the eigenvalues match the dense oracle to 1e-11."""
    A, B = problem(40, "c128", form="ph", seed=140 + nev)
    s = _solver(A, B)
    vals, vecs, nconv = s.solve(nev, tol=1e-12, ncv=ncv)
    _check_pairs("ph", A, B, 40, nev, vals, vecs, nconv)
    assert s.residuals().max() <= 1e-12
    s.close()


def test_batched_ncv_capped_at_nev_is_rejected():
    """N = {5, 200}, nev = 5: the smallest problem caps ncv at 5 = nev, which
    is the whole space of that problem but would let the larger one restart
    without adding a vector; the solve is refused with BSE_EINVAL."""
    from paper_2504_10096_gb300 import bse
    probs = [problem(n, "c128", form="ph", seed=150 + n) for n in (5, 200)]
    bs = bse.BatchedSolver([torch.from_numpy(a).cuda() for a, _ in probs],
                           [torch.from_numpy(b).cuda() for _, b in probs])
    rc, _, _ = bse.bse_solve_batched(bs.h, 2, 5, 1e-12)
    assert rc == bse.BSE_EINVAL
    bs.close()


@pytest.mark.parametrize("form", ["tda", "ph"])
def test_caller_ncv_equal_to_nev(form):
    # well-separated spectrum, so that one new vector per cycle converges in a few hundred steps
    n, nev = 60, 4
    rng = np.random.default_rng(77)
    G = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * 0.01
    A = np.diag(np.linspace(1.0, 3.0, n)) + (G + G.conj().T) / 2
    G = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * 0.01
    B = (G + G.T) / 2
    s = _solver(A, B if form == "ph" else None)
    vals, _, nconv = s.solve(nev, tol=1e-10, ncv=nev)
    ref = O.ph_lowest(A, B, nev)[0] if form == "ph" else O.tda_lowest(A, nev)[0]
    assert nconv == nev
    np.testing.assert_allclose(vals, ref, rtol=1e-9, atol=0)
    s.close()
