"""GPU parity of the three structure-preserving Lanczos variants (Sec. 2.2.1:
three variations of a structure-preserving thick-restart Lanczos) against the
dense FP64 oracle (zgeev of the full 2N matrix, Omega-normalised):

* Gruning: the Lanczos recurrence of H in the M inner product, even and odd
  bases, projected matrix with zero diagonal (eigenvalues +-omega);
* projected BSE: the folded recurrence with the projected problem solved as a
  small BSE matrix by the dense structure-preserving method;
* Shao (default) for reference on the same handles.

Sizes span several 128-row tiles with a ragged tail, the subspace close to and
equal to N (where the twin projections matter), N = 1 and N = 5, complex64
storage on the mixed path, a batch of uneven problems, and the config-4 recipe
at N = 4000 against its stored oracle eigenvalues."""
import os

import numpy as np
import pytest

import oracle as O
from tests.gpu_common import omega_metric_apply, problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
VARIANTS = ["gruning", "projected"]


def _variant(name):
    from paper_2504_10096_gb300 import bse
    return {"shao": bse.BSE_VARIANT_SHAO, "gruning": bse.BSE_VARIANT_GRUNING,
            "projected": bse.BSE_VARIANT_PROJECTED}[name]


def _solver(A, B, **kw):
    from paper_2504_10096_gb300 import bse
    return bse.Solver(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), **kw)


def _check(A, B, n, nev, vals, vecs, nconv, tol, rtol):
    om, Xo, Yo = O.ph_lowest(A, B, nev)
    assert nconv == nev
    np.testing.assert_allclose(vals, om, rtol=rtol, atol=0)
    Z = vecs.cpu().numpy().astype(np.complex128)
    res = O.relative_residuals_ph(A, B, vals, Z[:n], Z[n:])
    assert res.max() <= 10 * tol
    jn = np.real(np.einsum("ij,ij->j", Z.conj(), omega_metric_apply(Z)))
    np.testing.assert_allclose(jn, 1.0, atol=1e-6)
    gaps = np.diff(om)
    simple = np.ones(nev, bool)
    if nev > 1:
        simple[1:] &= gaps > 1e-4 * om[1:]
        simple[:-1] &= gaps > 1e-4 * om[:-1]
    ov = np.abs(np.einsum("ij,ij->j", Z.conj(), omega_metric_apply(np.vstack([Xo, Yo]))))
    np.testing.assert_allclose(ov[simple], 1.0, atol=1e-6)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n,nev,ncv", [(300, 10, 42), (515, 20, 0), (260, 12, 30)])
def test_variant_fp64_against_zgeev(variant, n, nev, ncv):
    A, B = problem(n, "c128", seed=700 + n)
    s = _solver(A, B)
    vals, vecs, nconv = s.solve(nev, tol=1e-12, ncv=ncv, variant=_variant(variant))
    _check(A, B, n, nev, vals, vecs, nconv, 1e-12, 1e-11)
    assert s.residuals().max() <= 1e-12
    s.close()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nev,ncv", [(10, 39), (38, 39), (10, 40), (39, 40), (40, 40)])
def test_variant_subspace_close_to_n(variant, nev, ncv):
    """N = 40 with ncv = N - 1 or N: the twin projections keep the second copy of
    every omega out of the basis, so every counted pair reaches tol."""
    A, B = problem(40, "c128", seed=140 + nev)
    s = _solver(A, B)
    vals, vecs, nconv = s.solve(nev, tol=1e-12, ncv=ncv, variant=_variant(variant))
    _check(A, B, 40, nev, vals, vecs, nconv, 1e-12, 1e-11)
    s.close()


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_tiny(variant):
    """N = 1 (closed form omega = sqrt(a^2 - |b|^2)) and N = 5 (whole space)."""
    a, b = 2.5, 0.7 * np.exp(0.3j)
    A = np.array([[a]], dtype=np.complex128)
    B = np.array([[b]], dtype=np.complex128)
    s = _solver(A, B)
    vals, vecs, nconv = s.solve(1, tol=1e-12, variant=_variant(variant))
    assert nconv == 1
    np.testing.assert_allclose(vals, [np.sqrt(a * a - abs(b) ** 2)], rtol=1e-13)
    s.close()
    A, B = problem(5, "c128", seed=5)
    s = _solver(A, B)
    vals, vecs, nconv = s.solve(5, tol=1e-12, variant=_variant(variant))
    _check(A, B, 5, 5, vals, vecs, nconv, 1e-12, 1e-11)
    s.close()


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_mixed_c64(variant):
    """complex64 storage on the mixed path (FP64 basis) reaches an FP64 residual
    of 1e-10 and matches the oracle on the same complex64 values."""
    A, B = problem(600, "c64", seed=77)
    s = _solver(A, B, mixed=True)
    vals, vecs, nconv = s.solve(16, tol=1e-10, variant=_variant(variant))
    A64, B64 = A.astype(np.complex128), B.astype(np.complex128)
    _check(A64, B64, 600, 16, vals, vecs, nconv, 1e-10, 1e-9)
    assert s.residuals().max() <= 1e-10
    s.close()


def test_variants_agree_and_switch_on_one_handle():
    """The three variants on one handle (graphs captured per variant) give the
    same eigenvalues; the Shao result is unchanged by the switches."""
    from paper_2504_10096_gb300 import bse
    A, B = problem(700, "c128", seed=91)
    s = _solver(A, B)
    v0, _, _ = s.solve(15, tol=1e-12, vectors=False)
    v1, _, n1 = s.solve(15, tol=1e-12, vectors=False, variant=bse.BSE_VARIANT_GRUNING)
    v2, _, n2 = s.solve(15, tol=1e-12, vectors=False, variant=bse.BSE_VARIANT_PROJECTED)
    v3, _, _ = s.solve(15, tol=1e-12, vectors=False)
    assert n1 == 15 and n2 == 15
    np.testing.assert_allclose(v1, v0, rtol=1e-12, atol=0)
    np.testing.assert_allclose(v2, v0, rtol=1e-12, atol=0)
    np.testing.assert_array_equal(v3, v0)
    s.close()


def test_variant_graph_and_stream_launches_identical():
    from paper_2504_10096_gb300 import bse
    A, B = problem(400, "c128", seed=13)
    s = _solver(A, B)
    a, _, _ = s.solve(10, tol=1e-12, vectors=False, variant=bse.BSE_VARIANT_GRUNING)
    b, _, _ = s.solve(10, tol=1e-12, vectors=False, variant=bse.BSE_VARIANT_GRUNING, graphs=False)
    np.testing.assert_array_equal(a, b)
    s.close()


def test_variant_invalid_and_tda():
    from paper_2504_10096_gb300 import bse
    A, B = problem(100, "c128", seed=3)
    s = _solver(A, B)
    with pytest.raises(bse.BSEError):
        s.solve(4, tol=1e-10, variant=3)
    s.close()
    A, _ = problem(120, "c128", form="tda", seed=4)
    t = bse.Solver(torch.from_numpy(A).cuda())
    ref = O.tda_lowest(A, 6)[0]
    for v in (bse.BSE_VARIANT_GRUNING, bse.BSE_VARIANT_PROJECTED):   # TDA: the plain recurrence
        vals, _, nconv = t.solve(6, tol=1e-12, vectors=False, variant=v)
        assert nconv == 6
        np.testing.assert_allclose(vals, ref, rtol=1e-12, atol=0)
    t.close()


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_batched_uneven(variant):
    from paper_2504_10096_gb300 import bse
    sizes = [130, 257, 400, 515]
    probs = [problem(n, "c64", seed=900 + n) for n in sizes]
    bs = bse.BatchedSolver([torch.from_numpy(a).cuda() for a, _ in probs],
                           [torch.from_numpy(b).cuda() for _, b in probs], mixed=True)
    vals, _, nconv = bs.solve(8, tol=1e-10, variant=_variant(variant))
    assert np.all(nconv == 8)
    for i, (a, b) in enumerate(probs):
        ref = O.ph_lowest(a.astype(np.complex128), b.astype(np.complex128), 8)[0]
        np.testing.assert_allclose(vals[i], ref, rtol=1e-9, atol=0)
        assert bs.residuals(i).max() <= 1e-10
    bs.close()


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_config4_recipe_n4000(variant):
    """Config-4 recipe (energies in [1, 12] eV, N_G = 2000) at N = 4000 on the
    mixed path at tol 1e-6: all 200 pairs within tol and the stored oracle
    eigenvalues to 1e-6 relative."""
    from paper_2504_10096_gb300 import bse
    from synthetic import make_problem, reduced_spec
    spec = reduced_spec(4, 4000)
    p = make_problem(spec)
    gold = np.loadtxt(os.path.join(GOLD, "config4r_omega.txt"))
    s = bse.Solver(torch.from_numpy(p["A"]).cuda(), torch.from_numpy(p["B"]).cuda(), mixed=True)
    vals, _, nconv = s.solve(spec.nev, tol=1e-6, vectors=False, variant=_variant(variant))
    assert nconv == spec.nev
    assert s.residuals().max() <= 1e-6
    np.testing.assert_allclose(vals, gold, rtol=1e-6, atol=0)
    st = s.stats()
    print(f"config-4 recipe N=4000 {variant}: steps {st['steps']}, restarts {st['restarts']}, "
          f"{st['ms_total']:.1f} ms")
    s.close()
