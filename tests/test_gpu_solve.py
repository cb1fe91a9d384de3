"""GPU parity of the iterative solver against the dense FP64 oracle.

Eigenvalues are unique and compared one by one; eigenvectors are unique up to
a phase and are compared through |z_gpu^H Omega z_oracle| (PH) or
|x_gpu^H x_oracle| (TDA), plus residuals and the Omega-normalisation."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import omega_metric_apply, problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _solver(A, B=None):
    from paper_2504_10096_gb300 import bse
    return bse.Solver(torch.from_numpy(A).cuda(), None if B is None else torch.from_numpy(B).cuda())


@pytest.mark.parametrize("n,nev", [(300, 8), (515, 12)])
def test_tda_fp64(n, nev):
    A, _ = problem(n, "c128", form="tda", seed=n)
    s = _solver(A)
    vals, vecs, nconv = s.solve(nev, tol=1e-12)
    lam, Xo = O.tda_lowest(A, nev)
    assert nconv == nev
    np.testing.assert_allclose(vals, lam, rtol=1e-10, atol=0)
    X = vecs.cpu().numpy()
    ov = np.abs(np.einsum("ij,ij->j", X.conj(), Xo))
    np.testing.assert_allclose(ov, 1.0, atol=1e-8)
    assert O.relative_residuals_tda(A, vals, X).max() < 1e-11
    assert s.stats()["max_residual"] < 1e-11
    s.close()


@pytest.mark.parametrize("n,nev", [(300, 10), (515, 16)])
def test_ph_fp64(n, nev):
    A, B = problem(n, "c128", seed=n + 1)
    s = _solver(A, B)
    vals, vecs, nconv = s.solve(nev, tol=1e-12)
    om, Xo, Yo = O.ph_lowest(A, B, nev)
    assert nconv == nev
    np.testing.assert_allclose(vals, om, rtol=1e-10, atol=0)
    Z = vecs.cpu().numpy()
    Zo = np.vstack([Xo, Yo])
    # Omega-normalisation and overlap with the oracle's vectors
    jn = np.real(np.einsum("ij,ij->j", Z.conj(), omega_metric_apply(Z)))
    np.testing.assert_allclose(jn, 1.0, atol=1e-10)
    ov = np.abs(np.einsum("ij,ij->j", Z.conj(), omega_metric_apply(Zo)))
    np.testing.assert_allclose(ov, 1.0, atol=1e-8)
    X, Y = Z[:n], Z[n:]
    assert O.relative_residuals_ph(A, B, vals, X, Y).max() < 1e-11
    # Eq. 7: the -omega partner (conj Y; conj X) needs no extra solve
    H = O.bse_hamiltonian(A, B)
    Zm = np.vstack([Y.conj(), X.conj()])
    assert np.linalg.norm(H @ Zm + Zm * vals) / np.linalg.norm(Zm) < 1e-10
    s.close()


def test_ph_c64_fp32_counts_only_pairs_below_tol():
    """BSE_C64 (FP32 storage, basis and products): the FP64 Rayleigh-quotient
    refinement gives eigenvalues to 1e-6; nconv counts exactly the returned
    pairs whose FP64 residual is <= tol (the FP32 floor is near eps_32 times
    the folded operator's spectral range, so some may miss a tight tol)."""
    from paper_2504_10096_gb300 import bse
    n, nev, tol = 600, 12, 1e-5
    A, B = problem(n, "c64", seed=17)
    s = _solver(A, B)
    vals, vecs, nconv = s.solve(nev, tol=tol, check=False)
    assert s.status in (bse.BSE_OK, bse.BSE_ENOCONV)
    res = s.residuals()
    assert nconv == int(np.sum(res <= tol))
    assert (s.status == bse.BSE_OK) == (nconv == nev)
    om, _, _ = O.ph_lowest(A.astype(np.complex128), B.astype(np.complex128), nev)
    np.testing.assert_allclose(vals, om, rtol=1e-6, atol=0)
    assert res.max() < 1e-4
    s.close()


def test_b_zero_equals_tda():
    """B = 0: the PH solve returns the TDA spectrum (Sec. 1)."""
    n, nev = 256, 6
    A, _ = problem(n, "c128", form="tda", seed=21)
    s = _solver(A, np.zeros_like(A))
    vals, _, _ = s.solve(nev, tol=1e-12)
    lam, _ = O.tda_lowest(A, nev)
    np.testing.assert_allclose(vals, lam, rtol=1e-10)
    s.close()


def test_diagonal_complex_coupling_closed_form():
    """A = diag(a), B = diag(b): omega_i = sqrt(a_i^2 - |b_i|^2) (decoupled 2x2)."""
    rng = np.random.default_rng(4)
    n, nev = 200, 7
    a = rng.uniform(1.5, 10.0, n)
    b = rng.uniform(0.0, 0.4, n) * np.exp(2j * np.pi * rng.uniform(size=n))
    s = _solver(np.diag(a).astype(np.complex128), np.diag(b))
    vals, _, _ = s.solve(nev, tol=1e-12)
    np.testing.assert_allclose(vals, np.sort(np.sqrt(a * a - np.abs(b) ** 2))[:nev], rtol=1e-10)
    s.close()


def test_degenerate_scalar_blocks():
    """A = aI, B = bI: every omega equals sqrt(a^2 - |b|^2); each Krylov chain
    breaks down at once and the solver restarts it with fresh vectors."""
    n, nev = 48, 5
    a, b = 2.0, 0.5 * np.exp(0.7j)
    s = _solver(a * np.eye(n, dtype=np.complex128), b * np.eye(n, dtype=np.complex128))
    vals, _, nconv = s.solve(nev, tol=1e-12)
    assert nconv == nev
    np.testing.assert_allclose(vals, np.sqrt(a * a - abs(b) ** 2), rtol=1e-12)
    s.close()


def test_not_positive_definite_is_reported():
    from paper_2504_10096_gb300 import bse
    n = 64
    A = np.eye(n, dtype=np.complex128)
    B = 2.0 * np.eye(n, dtype=np.complex128)
    s = _solver(A, B)
    with pytest.raises(bse.BSEError) as ei:
        s.solve(4, tol=1e-10)
    assert ei.value.status == bse.BSE_ENOTPD
    s.close()


def test_invalid_arguments():
    from paper_2504_10096_gb300 import bse
    A, B = problem(130, "c128", seed=2)
    s = _solver(A, B)
    rc, _, _ = bse.bse_solve(s.h, 0, 1e-10)
    assert rc == bse.BSE_EINVAL
    rc, _, _ = bse.bse_solve(s.h, 131, 1e-10)
    assert rc == bse.BSE_EINVAL
    assert bse.bse_backward(s.h, np.zeros(3).ctypes.data, bse.BSE_HOST, 1, 1) == bse.BSE_ESTATE
    s.close()


def test_config0_tda_n2000():
    """Workload config 0: TDA, N = 2000, lowest 20, FP64."""
    from synthetic import CONFIGS, make_problem
    spec = CONFIGS[0]
    p = make_problem(spec)
    s = _solver(p["A"])
    vals, vecs, nconv = s.solve(spec.nev, tol=1e-12)
    lam, _ = O.tda_lowest(p["A"], spec.nev)
    np.testing.assert_allclose(vals, lam, rtol=1e-10, atol=0)
    s.close()


@pytest.mark.parametrize("form", ["ph", "tda"])
def test_df64_products_solve(form):
    """BSE_C128_DF reaches the FP64-path tolerances (eigenvalues 1e-10)."""
    from paper_2504_10096_gb300 import bse
    n, nev = 515, 12
    A, B = problem(n, "c128", form=form, seed=77)
    s = bse.Solver(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda() if form == "ph" else None, df=True)
    vals, vecs, nconv = s.solve(nev, tol=1e-12)
    ref = O.ph_lowest(A, B, nev)[0] if form == "ph" else O.tda_lowest(A, nev)[0]
    assert nconv == nev
    np.testing.assert_allclose(vals, ref, rtol=1e-10, atol=0)
    assert s.stats()["max_residual"] < 1e-11
    s.close()


def test_mixed_c64_storage_reaches_fp64_class():
    """BSE_C64_MIXED: complex64 storage, FP64 basis, double-FP32 products --
    residuals far below what FP32 products allow (the folded operator
    squares the spectral range), eigenvalues at the FP64-path tolerance."""
    from paper_2504_10096_gb300 import bse
    n, nev = 600, 12
    A, B = problem(n, "c64", seed=19)
    s = bse.Solver(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), mixed=True)
    vals, vecs, nconv = s.solve(nev, tol=1e-10)
    om, Xo, Yo = O.ph_lowest(A.astype(np.complex128), B.astype(np.complex128), nev)
    assert nconv == nev
    np.testing.assert_allclose(vals, om, rtol=1e-10, atol=0)
    assert s.residuals().max() <= 1e-10
    Z = vecs.cpu().numpy().astype(np.complex128)
    assert vecs.dtype == torch.complex64
    ov = np.abs(np.einsum("ij,ij->j", Z.conj(), omega_metric_apply(np.vstack([Xo, Yo]))))
    np.testing.assert_allclose(ov, 1.0, atol=1e-6)
    s.close()


@pytest.mark.parametrize("form,dtype", [("ph", "c128"), ("tda", "c128"), ("ph", "c64")])
def test_graph_replay_matches_stream_launches(form, dtype):
    """The Krylov steps replayed as CUDA graphs run the same kernels in the
    same order as stream launches: identical eigenvalues, vectors, counters."""
    A, B = problem(700, dtype, form=form, seed=77)
    s = _solver(A, B if form == "ph" else None)
    tol = 1e-12 if dtype == "c128" else 1e-6
    v1, z1, _ = s.solve(12, tol=tol, graphs=False, check=False)
    st1 = s.stats()
    v2, z2, _ = s.solve(12, tol=tol, graphs=True, persistent=False, check=False)
    st2 = s.stats()
    v3, z3, _ = s.solve(12, tol=tol, graphs=True, persistent=False, check=False)   # graphs from the cache
    st3 = s.stats()
    assert np.array_equal(v1, v2) and np.array_equal(v2, v3)
    assert torch.equal(z1, z2) and torch.equal(z2, z3)
    for k in ("steps", "passes", "restarts", "launches"):
        assert st1[k] == st2[k] == st3[k], k
    assert st2["ms_product"] > 0.0 and st3["ms_product"] > 0.0
    s.close()


@pytest.mark.parametrize("form,dtype,n", [("ph", "c128", 700), ("tda", "c128", 700), ("ph", "c64", 700),
                                          ("tda", "c128", 2000), ("ph", "c128", 4000), ("tda", "c64", 3000)])
def test_persistent_steps_match_per_phase_kernels(form, dtype, n):
    """One small problem: the Krylov steps of a cycle run as one persistent cooperative
    launch (phases at a grid barrier) and give the same bits as the per-phase kernels
    (graphs and stream launches), with far fewer launches; N = 4000 and 3000 take the
    multi-row-block norm path of the persistent kernel."""
    A, B = problem(n, dtype, form=form, seed=91)
    s = _solver(A, B if form == "ph" else None)
    tol = 1e-12 if dtype == "c128" else 1e-6
    v1, z1, n1 = s.solve(12, tol=tol, graphs=False, check=False)
    st1 = s.stats()
    v2, z2, _ = s.solve(12, tol=tol, graphs=True, persistent=True, check=False)
    st2 = s.stats()
    v3, z3, _ = s.solve(12, tol=tol, graphs=True, persistent=True, check=False)
    assert n1 == 12 or dtype == "c64"
    assert np.array_equal(v1, v2) and np.array_equal(v2, v3)
    assert torch.equal(z1, z2) and torch.equal(z2, z3)
    for k in ("steps", "passes", "restarts"):
        assert st1[k] == st2[k], k
    assert st2["launches"] < st1["launches"] / 3, (st2["launches"], st1["launches"])
    s.close()


def test_product_shape_tuner():
    """The first solve of a handle times the candidate launch shapes on its
    own products and keeps the fastest; a second handle of the same kind is
    tuned from the process cache at creation.  The tile results do not depend
    on the shape, so both give bit-identical eigenpairs."""
    A, B = problem(900, "c128", seed=79)
    s1 = _solver(A, B)
    v1, z1, _ = s1.solve(10, tol=1e-12)
    st1 = s1.stats()
    assert st1["tuned"] == 1
    assert st1["shape_ctas_per_sm"] >= -1 and st1["shape_strided"] in (0, 1)
    s2 = _solver(A, B)
    v2, z2, _ = s2.solve(10, tol=1e-12)
    st2 = s2.stats()
    assert st2["tuned"] == 1
    assert (st2["shape_ctas_per_sm"], st2["shape_strided"]) == (st1["shape_ctas_per_sm"], st1["shape_strided"])
    assert np.array_equal(v1, v2) and torch.equal(z1, z2)
    s1.close()
    s2.close()


def test_graphs_follow_a_change_of_subspace_size():
    """Solves of different nev (hence ncv) on one handle: the step graphs are
    recaptured for the new size and the results match a fresh handle's."""
    A, B = problem(600, "c128", seed=83)
    s = _solver(A, B)
    v8, _, _ = s.solve(8, tol=1e-12)
    v14, _, _ = s.solve(14, tol=1e-12)
    v8b, _, _ = s.solve(8, tol=1e-12)
    s.close()
    f = _solver(A, B)
    w14, _, _ = f.solve(14, tol=1e-12)
    f.close()
    om, _, _ = O.ph_lowest(A, B, 14)
    np.testing.assert_allclose(v14, om, rtol=1e-10)
    np.testing.assert_allclose(v8, om[:8], rtol=1e-10)
    assert np.array_equal(v8, v8b)
    assert np.array_equal(v14, w14)
