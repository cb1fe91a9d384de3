"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formula: each checks it against a
closed form, an invariant stated in the paper (Sec. 1, Sec. 2.1.1, Eq. 7), an
independent algorithm (characteristic polynomial by Faddeev-LeVerrier, the
paper's Shao reduction against zgeev), or central finite differences.
"""
import numpy as np
import pytest

import oracle as O
from synthetic import BSEProblemSpec, make_problem

RNG = np.random.default_rng(20250414)


def rand_herm(n, rng, shift=0.0, scale=1.0):
    x = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * scale
    h = (x + x.conj().T) / 2
    return h + shift * np.eye(n)


def rand_sym(n, rng, scale=1.0):
    x = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * scale
    return (x + x.T) / 2


def pd_problem(n, rng, bscale=0.05):
    """A with spectrum in ~[2, 4], small complex symmetric B: M > 0."""
    A = rand_herm(n, rng, shift=3.0, scale=0.5 / np.sqrt(n))
    B = rand_sym(n, rng, scale=bscale / np.sqrt(n))
    return A, B


# ------------------------------------------------------------------ closed forms
def test_b_zero_reduces_to_tda():
    """B = 0: the PH spectrum is +-eig(A), i.e. the TDA result (Sec. 1)."""
    A = rand_herm(12, RNG, shift=3.0, scale=0.3)
    om, X, Y = O.ph_lowest(A, np.zeros_like(A), 12)
    lam, _ = O.tda_lowest(A, 12)
    np.testing.assert_allclose(om, lam, rtol=1e-13)
    assert np.abs(Y).max() < 1e-12
    full = O.ph_full_spectrum(A, np.zeros_like(A)).real
    np.testing.assert_allclose(np.sort(full), np.sort(np.concatenate([-lam, lam])), atol=1e-12)


def test_diagonal_a_b_zero_gives_diag():
    a = np.sort(RNG.uniform(1.5, 10, 9))
    A = np.diag(a).astype(complex)
    om, _, _ = O.ph_lowest(A, np.zeros_like(A), 9)
    np.testing.assert_allclose(om, a, rtol=1e-14)
    lam, X = O.tda_lowest(A, 9)
    np.testing.assert_allclose(lam, a, rtol=1e-14)


def test_scalar_blocks_closed_form():
    """A = aI, B = bI (b complex): omega = sqrt(a^2 - |b|^2), multiplicity N."""
    a, b = 2.5, 0.7 * np.exp(0.3j)
    n = 7
    A = a * np.eye(n, dtype=complex)
    B = b * np.eye(n, dtype=complex)
    om, X, Y = O.ph_lowest(A, B, n)
    np.testing.assert_allclose(om, np.sqrt(a * a - abs(b) ** 2) * np.ones(n), rtol=1e-13)
    lam = O.ph_lowest_shao(A, B, n)
    np.testing.assert_allclose(lam, np.sqrt(a * a - abs(b) ** 2) * np.ones(n), rtol=1e-13)


def test_diagonal_complex_coupling_closed_form():
    """A = diag(a_i), B = diag(b_i): N decoupled 2x2 blocks [[a, b], [-conj b, -a]]
    with omega_i = sqrt(a_i^2 - |b_i|^2).  A wrong conjugation or sign in the
    lower blocks of Eq. 1 gives a^2 - b^2 instead and fails here."""
    a = np.array([1.7, 2.2, 3.1, 4.0, 5.5])
    b = np.array([0.3 + 0.4j, -0.2 + 0.9j, 1.1j, 0.5 - 0.5j, -0.1])
    om, X, Y = O.ph_lowest(np.diag(a).astype(complex), np.diag(b), 5)
    ref = np.sort(np.sqrt(a * a - np.abs(b) ** 2))
    np.testing.assert_allclose(om, ref, rtol=1e-13)
    lam = O.ph_lowest_shao(np.diag(a).astype(complex), np.diag(b), 5)
    np.testing.assert_allclose(lam, ref, rtol=1e-13)


def test_real_blocks_closed_form():
    """Real A, B: omega^2 = eig((A - B)(A + B))."""
    n = 10
    x = RNG.standard_normal((n, n))
    A = (x + x.T) / 4 + 3 * np.eye(n)
    y = RNG.standard_normal((n, n))
    B = (y + y.T) / 10
    om, _, _ = O.ph_lowest(A.astype(complex), B.astype(complex), n)
    w2 = np.sort(np.linalg.eigvals((A - B) @ (A + B)).real)
    np.testing.assert_allclose(om ** 2, w2, rtol=1e-12)


def test_scalar_n1():
    a, b = 1.9, 0.4 - 0.8j
    om, X, Y = O.ph_lowest(np.array([[a]], complex), np.array([[b]]), 1)
    assert abs(om[0] - np.sqrt(a * a - abs(b) ** 2)) < 1e-14
    # J-normalisation |X|^2 - |Y|^2 = 1
    assert abs(abs(X[0, 0]) ** 2 - abs(Y[0, 0]) ** 2 - 1) < 1e-13


# ------------------------------------------------------------------ brute force
def _charpoly_faddeev_leverrier(M):
    """Coefficients of det(lambda I - M), highest first, from traces only."""
    n = M.shape[0]
    c = np.zeros(n + 1, dtype=complex)
    c[0] = 1.0
    Mk = np.zeros_like(M)
    for k in range(1, n + 1):
        Mk = M @ Mk + c[k - 1] * np.eye(n)
        c[k] = -np.trace(M @ Mk) / k
    return c


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_brute_force_characteristic_polynomial(n):
    rng = np.random.default_rng(100 + n)
    A, B = pd_problem(n, rng, bscale=0.4)
    H = O.bse_hamiltonian(A, B)
    roots = np.roots(_charpoly_faddeev_leverrier(H))
    pos = np.sort(roots.real[roots.real > 0])
    om, _, _ = O.ph_lowest(A, B, n)
    np.testing.assert_allclose(om, pos, rtol=1e-9)
    assert np.max(np.abs(roots.imag)) < 1e-8


# ------------------------------------------------------------------ invariants
@pytest.fixture(scope="module")
def pd40():
    rng = np.random.default_rng(7)
    A, B = pd_problem(40, rng, bscale=0.3)
    om, X, Y = O.ph_lowest(A, B, 40)
    return A, B, om, X, Y


def test_positive_definite_and_real_spectrum(pd40):
    A, B, om, X, Y = pd40
    assert O.is_positive_definite(A, B)
    full = O.ph_full_spectrum(A, B)
    assert np.max(np.abs(full.imag)) < 1e-10          # Sec. 1: real spectrum
    np.testing.assert_allclose(np.sort(full.real), np.sort(-full.real), atol=1e-11)  # +-omega


def test_eq7_eigenvector_relations(pd40):
    """Right/left eigenvectors for +omega and -omega (Eq. 7)."""
    A, B, om, X, Y = pd40
    H = O.bse_hamiltonian(A, B)
    Z = np.vstack([X, Y])
    np.testing.assert_allclose(H @ Z, Z * om, atol=1e-11)
    L = np.vstack([X, -Y])                      # left for +omega: L^H H = omega L^H
    np.testing.assert_allclose(L.conj().T @ H, om[:, None] * L.conj().T, atol=1e-11)
    Zm = np.vstack([Y.conj(), X.conj()])        # right for -omega
    np.testing.assert_allclose(H @ Zm, -Zm * om, atol=1e-11)
    Lm = np.vstack([-Y.conj(), X.conj()])       # left for -omega
    np.testing.assert_allclose(Lm.conj().T @ H, -om[:, None] * Lm.conj().T, atol=1e-11)


def test_j_orthonormality(pd40):
    A, B, om, X, Y = pd40
    Z = np.vstack([X, Y])
    G = Z.conj().T @ O.omega_metric(40) @ Z
    np.testing.assert_allclose(G, np.eye(40), atol=1e-10)


def test_shao_reduction_matches_zgeev(pd40):
    """Sec. 2.1.1: Q^dagger H Q = -i J M_r (Eqs. 4-5); M > 0 => M_r > 0;
    -iW Hermitian with eigenvalues +-omega (Eq. 6)."""
    A, B, om, X, Y = pd40
    n = 40
    Q = O.shao_q(n)
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(2 * n), atol=1e-14)
    Mr = O.shao_real_matrix(A, B)
    np.testing.assert_allclose(Q.conj().T @ O.bse_hamiltonian(A, B) @ Q,
                               -1j * O.shao_j(n) @ Mr, atol=1e-12)
    np.testing.assert_allclose(Mr, Mr.T, atol=0)
    assert np.linalg.eigvalsh(Mr)[0] > 0
    W, L = O.shao_skew_matrix(A, B)
    np.testing.assert_allclose(W, -W.T, atol=1e-12)
    lam, Xs, Ys = O.ph_lowest_shao(A, B, 10, vectors=True)
    np.testing.assert_allclose(lam, om[:10], rtol=1e-12)
    res = O.relative_residuals_ph(A, B, lam, Xs, Ys)
    assert res.max() < 1e-12
    # same eigenvectors up to a phase: |z_s^H Omega z| = 1
    Zs = np.vstack([Xs, Ys])
    Z = np.vstack([X[:, :10], Y[:, :10]])
    ov = np.abs(np.einsum("ij,ij->j", Zs.conj(), O.omega_metric(n) @ Z))
    np.testing.assert_allclose(ov, 1.0, atol=1e-9)


def test_degeneracy_preserved():
    """Structure-preserving solvers keep degeneracies (Sec. 2.1.1): a problem
    built as two identical uncoupled copies has every omega exactly doubled."""
    rng = np.random.default_rng(3)
    A1, B1 = pd_problem(6, rng, bscale=0.3)
    Z0 = np.zeros_like(A1)
    A = np.block([[A1, Z0], [Z0, A1]])
    B = np.block([[B1, Z0], [Z0, B1]])
    lam = O.ph_lowest_shao(A, B, 12)
    np.testing.assert_allclose(lam[0::2], lam[1::2], rtol=1e-12)


def test_folded_operator_identities(pd40):
    """The real-linear halves used by the GPU path: with u = X + conj(Y),
    M+ u = omega (X - conj(Y)), M- M+ u = omega^2 u, and
    |X|^2 - |Y|^2 = Re(u^H M+ u) / omega."""
    A, B, om, X, Y = pd40
    U = X + Y.conj()
    P = O.apply_mplus(A, B, U)
    np.testing.assert_allclose(P, (X - Y.conj()) * om, atol=1e-11)
    np.testing.assert_allclose(O.apply_mminus(A, B, P), U * om ** 2, atol=1e-10)
    jn = np.sum(np.abs(X) ** 2, 0) - np.sum(np.abs(Y) ** 2, 0)
    np.testing.assert_allclose(jn, np.real(np.sum(U.conj() * P, 0)) / om, rtol=1e-11)
    # the i * M+ u image ("twin") is an eigenvector of M- M+ as well
    T = 1j * P
    np.testing.assert_allclose(O.apply_mminus(A, B, O.apply_mplus(A, B, T)), T * om ** 2, atol=1e-10)


@pytest.mark.parametrize("sign", [1, -1])
def test_real_form_of_the_folded_halves(sign):
    """Eq. 5 form used by the product kernels: on (Re u, Im u) the map
    u -> A u + s B conj(u) is the real matrix [[U_re, -V_im], [U_im, V_re]] with
    U = A + sB, V = A - sB (for s = +1 the paper's M_r up to y -> -y), and the
    transpose use of a stored block (A = A^H, B = B^T) is [[U_re, U_im], [-V_im, V_re]]."""
    rng = np.random.default_rng(11)
    n = 7
    A = rand_herm(n, rng, shift=2.0)
    B = rand_sym(n, rng, scale=0.3)
    U, V = A + sign * B, A - sign * B
    R = np.block([[U.real, -V.imag], [U.imag, V.real]])
    apply = O.apply_mplus if sign > 0 else O.apply_mminus
    for _ in range(3):
        u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        w = apply(A, B, u)
        np.testing.assert_allclose(R @ np.r_[u.real, u.imag], np.r_[w.real, w.imag], atol=1e-12)
    # transpose use: column block of a stored tile acting on the row block's entries
    RT = np.block([[U.real.T, U.imag.T], [-V.imag.T, V.real.T]])
    np.testing.assert_allclose(RT, R.T, atol=0)
    # the real matrix is symmetric (M+/M- self-adjoint for Re(x^H y)), and for s = +1 it is
    # positive definite exactly when M of Eq. 2 is
    np.testing.assert_allclose(R, R.T, atol=1e-12)
    if sign > 0:
        assert (np.linalg.eigvalsh(R).min() > 0) == O.is_positive_definite(A, B)
        # and a B large enough to break positive definiteness breaks both the same way
        Bbig = 4.0 * B / np.linalg.norm(B, 2) * np.linalg.eigvalsh(A).min()
        Ub, Vb = A + Bbig, A - Bbig
        Rb = np.block([[Ub.real, -Vb.imag], [Ub.imag, Vb.real]])
        assert (np.linalg.eigvalsh(Rb).min() > 0) == O.is_positive_definite(A, Bbig)


def test_apply_bse_block_form(pd40):
    """H X from the two stored blocks: Y1 = A X1 + B X2, Y2 = -conj(A conj X2 + B conj X1)."""
    A, B = pd40[0], pd40[1]
    Xr = RNG.standard_normal((80, 3)) + 1j * RNG.standard_normal((80, 3))
    Y = O.apply_bse(A, B, Xr)
    x1, x2 = Xr[:40], Xr[40:]
    np.testing.assert_allclose(Y[:40], A @ x1 + B @ x2, atol=1e-12)
    np.testing.assert_allclose(Y[40:], -(A @ x2.conj() + B @ x1.conj()).conj(), atol=1e-12)


def test_metric_matrix_eq3(pd40):
    """Eq. 3: H = Omega M with M Hermitian (Eq. 2)."""
    A, B = pd40[0], pd40[1]
    M = O.metric_matrix(A, B)
    np.testing.assert_allclose(M, M.conj().T, atol=0)
    np.testing.assert_allclose(O.omega_metric(40) @ M, O.bse_hamiltonian(A, B), atol=0)


# ------------------------------------------------------------------ residuals and Rayleigh quotients
def test_omega_rayleigh_quotient_n1_closed_form():
    """N = 1, H = [[a, b], [-conj b, -a]], z = (x; y): written out by hand,
    z^H Omega H z = a(|x|^2 + |y|^2) + 2 Re(conj(x) b y) and z^H Omega z = |x|^2 - |y|^2."""
    a, b = 2.3, 0.6 * np.exp(0.7j)
    x = RNG.standard_normal((1, 5)) + 1j * RNG.standard_normal((1, 5))
    y = 0.5 * (RNG.standard_normal((1, 5)) + 1j * RNG.standard_normal((1, 5)))
    rho = O.j_rayleigh_quotients(np.array([[a]]), np.array([[b]]), x, y)
    want = (a * (abs(x) ** 2 + abs(y) ** 2) + 2 * np.real(x.conj() * b * y)) / (abs(x) ** 2 - abs(y) ** 2)
    np.testing.assert_allclose(rho, want[0], rtol=1e-14)
    # on the eigenvector (a - w) x + b y = 0 it is w = sqrt(a^2 - |b|^2) (Sec. 1)
    w = np.sqrt(a * a - abs(b) ** 2)
    xe = np.array([[1.0 + 0.2j]])
    ye = -(a - w) * xe / b
    np.testing.assert_allclose(O.j_rayleigh_quotients(np.array([[a]]), np.array([[b]]), xe, ye), [w], rtol=1e-14)


def test_omega_rayleigh_quotient_is_second_order(pd40):
    """z^H M z / z^H Omega z is stationary at the eigenvectors of H = Omega M:
    an O(eps) error in z gives an O(eps^2) error in omega."""
    A, B, om, X, Y = pd40
    rng = np.random.default_rng(3)
    d = rng.standard_normal((80, 5)) + 1j * rng.standard_normal((80, 5))
    d /= np.linalg.norm(d, axis=0)
    err = []
    for eps in (1e-3, 1e-4):
        Z = np.vstack([X[:, :5], Y[:, :5]]) + eps * d
        err.append(np.max(np.abs(O.j_rayleigh_quotients(A, B, Z[:40], Z[40:]) - om[:5])))
    assert err[0] < 1e-4 and err[1] < err[0] / 50


def test_relative_residuals_closed_forms(pd40):
    """Exact pairs give ~0; a shift w -> w + delta gives exactly |delta| / |w + delta|
    (H z - (w + delta) z = -delta z); the value does not depend on the scaling of z;
    N = 1, z = (1; 0): ||(a - w, -conj b)|| / w."""
    A, B, om, X, Y = pd40
    assert np.max(O.relative_residuals_ph(A, B, om, X, Y)) < 1e-12
    delta = 1e-3 * om
    c = 2.5 * np.exp(1.1j)
    r = O.relative_residuals_ph(A, B, om + delta, c * X, c * Y)
    np.testing.assert_allclose(r, np.abs(delta) / np.abs(om + delta), rtol=1e-8)
    a, b = 2.3, 0.6 * np.exp(0.7j)
    w = np.sqrt(a * a - abs(b) ** 2)
    r1 = O.relative_residuals_ph(np.array([[a]]), np.array([[b]]), np.array([w]),
                                 np.array([[1.0]]), np.array([[0.0]]))
    np.testing.assert_allclose(r1, [np.hypot(a - w, abs(b)) / w], rtol=1e-14)
    # TDA: diagonal A, x = e1 + e2 (not an eigenvector)
    lam, x = 1.7, np.zeros((3, 1), complex)
    x[0, 0] = x[1, 0] = 1.0
    At = np.diag([1.0, 2.0, 3.0]).astype(complex)
    rt = O.relative_residuals_tda(At, np.array([lam]), x)
    np.testing.assert_allclose(rt, [np.hypot(1.0 - lam, 2.0 - lam) / (lam * np.sqrt(2.0))], rtol=1e-14)
    lt, Xt = O.tda_lowest(A, 6)
    assert np.max(O.relative_residuals_tda(A, lt, Xt)) < 1e-13


# ------------------------------------------------------------------ gradients (FD)
def _fd_dirs(n, rng, count):
    out = []
    for _ in range(count):
        i, j = rng.integers(0, n, 2)
        out.append((int(i), int(j)))
    return out


def test_hf_gradient_ph_against_finite_differences():
    """Central FD of L = sum g_i omega_i through zgeev against G_A, G_B (the
    seven Hermitian / symmetric perturbation directions)."""
    rng = np.random.default_rng(11)
    n, k = 8, 4
    A, B = pd_problem(n, rng, bscale=0.4)
    g = rng.uniform(0.2, 1.0, k)
    om, X, Y = O.ph_lowest(A, B, k)
    GA, GB = O.hf_gradient_ph(X, Y, g)
    np.testing.assert_allclose(GA, GA.conj().T, atol=1e-13)
    np.testing.assert_allclose(GB, GB.T, atol=1e-13)

    def loss(a, b):
        return float(np.dot(g, O.ph_lowest(a, b, k)[0]))

    h = 1e-5
    for (i, j) in _fd_dirs(n, rng, 6):
        if i == j:
            cases = [("A", np.outer(np.eye(n)[i], np.eye(n)[i]), GA[i, i].real),
                     ("B", np.outer(np.eye(n)[i], np.eye(n)[i]), GB[i, i].real),
                     ("B", 1j * np.outer(np.eye(n)[i], np.eye(n)[i]), GB[i, i].imag)]
        else:
            eij = np.outer(np.eye(n)[i], np.eye(n)[j])
            cases = [("A", eij + eij.T, 2 * GA[i, j].real),
                     ("A", 1j * (eij - eij.T), 2 * GA[i, j].imag),
                     ("B", eij + eij.T, 2 * GB[i, j].real),
                     ("B", 1j * (eij + eij.T), 2 * GB[i, j].imag)]
        for which, E, ref in cases:
            if which == "A":
                fd = (loss(A + h * E, B) - loss(A - h * E, B)) / (2 * h)
            else:
                fd = (loss(A, B + h * E) - loss(A, B - h * E)) / (2 * h)
            assert abs(fd - ref) < 1e-7, (which, i, j, fd, ref)


def test_hf_gradient_tda_against_finite_differences():
    rng = np.random.default_rng(12)
    n, k = 9, 3
    A = rand_herm(n, rng, shift=3.0, scale=0.5)
    g = rng.uniform(0.2, 1.0, k)
    lam, X = O.tda_lowest(A, k)
    GA = O.hf_gradient_tda(X, g)

    def loss(a):
        return float(np.dot(g, O.tda_lowest(a, k)[0]))

    h = 1e-5
    for (i, j) in _fd_dirs(n, rng, 5):
        eij = np.outer(np.eye(n)[i], np.eye(n)[j])
        if i == j:
            cases = [(eij, GA[i, i].real)]
        else:
            cases = [(eij + eij.T, 2 * GA[i, j].real), (1j * (eij - eij.T), 2 * GA[i, j].imag)]
        for E, ref in cases:
            fd = (loss(A + h * E) - loss(A - h * E)) / (2 * h)
            assert abs(fd - ref) < 1e-7


# ------------------------------------------------------------------ generator
def test_generator_structure_and_norms():
    spec = BSEProblemSpec(n=300, n_g=60, seed=9)
    p = make_problem(spec)
    A, B = p["A"], p["B"]
    assert np.array_equal(A, A.conj().T)
    assert np.array_equal(B, B.T)
    assert np.all(A.diagonal().imag == 0)
    # ||K_x - W||, ||B||: B's 2-norm hits the spec
    assert abs(np.linalg.norm(B, 2) - 0.15) < 1e-10
    off = A - np.diag(p["energies"])
    assert np.linalg.norm(off, 2) <= 0.3 + 0.2 + 1e-9
    assert O.is_positive_definite(A, B)
    # determinism: same seed, same bytes
    q = make_problem(spec)
    assert np.array_equal(q["A"], A) and np.array_equal(q["B"], B)


def test_generator_c64_storage_is_exact():
    p = make_problem(BSEProblemSpec(n=200, n_g=40, seed=2, dtype="c64"))
    A, B = p["A"], p["B"]
    assert A.dtype == np.complex64 and B.dtype == np.complex64
    assert np.array_equal(A, A.conj().T) and np.array_equal(B, B.T)


def test_g_vectors_order():
    from synthetic import g_vectors
    g = g_vectors(27)
    n2 = (g * g).sum(1)
    assert n2[0] == 0 and np.all(np.diff(n2) >= 0)
    assert len({tuple(x) for x in g}) == 27
    assert (n2 == 1).sum() == 6 and (n2 == 2).sum() == 12 and (n2 == 3).sum() == 8
