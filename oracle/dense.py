"""FP64 dense oracle for the Bethe-Salpeter eigenproblem.

TEST INFRASTRUCTURE ONLY.  This module is imported by tests/, by
__graft_entry__.smoke() and by bench.py's cpu_baseline / reference leg.  The
product path (the CUDA library and its Python binding) never imports, links or
executes anything here, and this module imports nothing from the product path.

It computes, slowly and plainly, what the iterative GPU solver must reach:

* the Tamm-Dancoff (TDA) form: lowest eigenpairs of the Hermitian block A
  (the C = 0 case of Sec. 1, after Eq. 3), by dense zheevd;
* the pseudo-Hermitian form H = [[A, B], [-conj(B), -conj(A)]] (Eq. 1 with
  R = A, C = B and, in the optical case of Sec. 1, anti-resonant block
  conj(R) and C = C^T): lowest positive eigenvalues and right eigenvectors
  by dense zgeev of the full 2N x 2N matrix, normalised so that
  z^H Omega z = 1 with Omega = diag(I, -I) (Eq. 2);
* the same positive eigenvalues by the paper's own dense reduction (Sec. 2.1.1,
  Eqs. 4-6): real symmetric M_r, Cholesky M_r = L L^T, real skew-symmetric
  W = L^T J L, and the Hermitian matrix -iW whose eigenvalues are +-omega;
* the plain operator definitions the GPU path applies (H X, and the two
  real-linear halves M+ u = A u + B conj(u), M- w = A w - B conj(w));
* Hellmann-Feynman gradients of eigenvalues with respect to A and B, from the
  left eigenvector Omega z of Eq. 7.

Every function is FP64 / complex128 regardless of the storage type of the
inputs.  All parity of every function here is pinned by tests/test_oracle_pins.py
against closed forms, invariants, brute force and finite differences.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

__all__ = [
    "bse_hamiltonian",
    "metric_matrix",
    "omega_metric",
    "is_positive_definite",
    "tda_lowest",
    "ph_full_spectrum",
    "ph_lowest",
    "shao_q",
    "shao_j",
    "shao_real_matrix",
    "shao_skew_matrix",
    "ph_lowest_shao",
    "apply_bse",
    "apply_a",
    "apply_mplus",
    "apply_mminus",
    "hf_gradient_tda",
    "hf_gradient_ph",
    "relative_residuals_ph",
    "relative_residuals_tda",
    "j_rayleigh_quotients",
]


def _c128(x):
    return np.asarray(x, dtype=np.complex128)


# ---------------------------------------------------------------- definitions
def bse_hamiltonian(A, B):
    """H = [[A, B], [-conj(B), -conj(A)]]: Eq. 1 in the optical case (Sec. 1),
    R = A Hermitian, C = B = B^T, so -C^dagger = -conj(B) and the
    anti-resonant block is conj(A)."""
    A = _c128(A)
    B = np.zeros_like(A) if B is None else _c128(B)
    return np.block([[A, B], [-B.conj(), -A.conj()]])


def metric_matrix(A, B):
    """M = [[A, B], [B^dagger, conj(A)]] of Eq. 2, with H = Omega M (Eq. 3)."""
    A = _c128(A)
    B = np.zeros_like(A) if B is None else _c128(B)
    return np.block([[A, B], [B.conj().T, A.conj()]])


def omega_metric(n):
    """Omega = diag(I, -I) of Eq. 2 (often written J; the paper's J is the skew matrix of Eq. 4)."""
    return np.diag(np.concatenate([np.ones(n), -np.ones(n)]))


def is_positive_definite(A, B) -> bool:
    """Cholesky test of M (Sec. 1: M positive definite <=> Hermitian-definite
    generalised problem with real spectrum)."""
    try:
        np.linalg.cholesky(metric_matrix(A, B))
        return True
    except np.linalg.LinAlgError:
        return False


# ---------------------------------------------------------------- TDA oracle
def tda_lowest(A, nev):
    """Lowest nev eigenpairs of the Hermitian A (TDA, C = 0; Sec. 1 and the
    resonant-only runs of Sec. 3), dense zheevd.  Returns (lam, X) ascending,
    columns of X unit 2-norm."""
    A = _c128(A)
    lam, X = sla.eigh(A, driver="evd")
    return lam[:nev], X[:, :nev]


# ---------------------------------------------------------------- PH oracle
def ph_full_spectrum(A, B):
    """All 2N eigenvalues of H (dense zgeev), ascending by real part."""
    ev = sla.eigvals(bse_hamiltonian(A, B))
    return ev[np.argsort(ev.real)]


def ph_lowest(A, B, nev, imag_tol=1e-8):
    """Lowest nev positive eigenvalues omega of H with right eigenvectors
    z = (X; Y) normalised to z^H Omega z = 1 (Eqs. 1-3, Eq. 7), by dense zgeev.

    Raises ValueError if an eigenvalue has |Im| above imag_tol * ||H||_F, i.e.
    the spectrum is not real (Sec. 1: M is then not positive definite)."""
    A = _c128(A)
    n = A.shape[0]
    H = bse_hamiltonian(A, B)
    ev, Z = sla.eig(H)
    scale = np.linalg.norm(H)
    if np.max(np.abs(ev.imag)) > imag_tol * scale:
        raise ValueError("spectrum of H is not real: M is not positive definite")
    pos = np.where(ev.real > 0)[0]
    pos = pos[np.argsort(ev.real[pos])][:nev]
    omega = ev.real[pos]
    Z = Z[:, pos]
    J = omega_metric(n)
    # J-normalisation: z^H Omega z > 0 for the positive branch when M > 0
    jn = np.real(np.einsum("ij,ij->j", Z.conj(), J @ Z))
    if np.any(jn <= 0):
        raise ValueError("non-positive J-norm on the positive branch")
    Z = Z / np.sqrt(jn)
    # fix the arbitrary phase: largest |X_i| real positive (cosmetic only)
    X = Z[:n]
    k = np.argmax(np.abs(X), axis=0)
    ph = X[k, np.arange(X.shape[1])]
    Z = Z * (np.abs(ph) / ph)
    return omega, Z[:n], Z[n:]


def shao_q(n):
    """Unitary Q of Eq. 4: (1/sqrt 2) [[I, -iI], [I, iI]]."""
    I = np.eye(n)
    return np.block([[I, -1j * I], [I, 1j * I]]) / np.sqrt(2.0)


def shao_j(n):
    """Real skew-symmetric J of Eq. 4 (not the metric Omega of Eq. 2)."""
    I = np.eye(n)
    Z = np.zeros((n, n))
    return np.block([[Z, I], [-I, Z]])


def shao_real_matrix(A, B):
    """M_r of Eq. 5 with R = A, C = B:
    [[Re(A+B), Im(A-B)], [-Im(A+B), Re(A-B)]]."""
    A = _c128(A)
    B = np.zeros_like(A) if B is None else _c128(B)
    return np.block([[(A + B).real, (A - B).imag], [-(A + B).imag, (A - B).real]])


def shao_skew_matrix(A, B):
    """W = L^T J L with M_r = L L^T (Sec. 2.1.1, before Eq. 6); returns (W, L)."""
    Mr = shao_real_matrix(A, B)
    L = np.linalg.cholesky(Mr)
    n = _c128(A).shape[0]
    W = L.T @ shao_j(n) @ L
    return W, L


def ph_lowest_shao(A, B, nev, vectors=False):
    """Lowest nev positive eigenvalues of H through the paper's dense reduction
    (Sec. 2.1.1, Eqs. 4-6): -iW is Hermitian with eigenvalues +-omega.

    With vectors=True also returns J-normalised right eigenvectors, recovered
    from q (eigenvector of -iW) as y = L^{-T} q, z = Q y: from
    Q^dagger H Q = -i J M_r and M_r = L L^T one gets -iW (L^T y) = omega (L^T y)."""
    A = _c128(A)
    n = A.shape[0]
    W, L = shao_skew_matrix(A, B)
    Hh = -1j * W
    if not vectors:
        lam = sla.eigh(Hh, eigvals_only=True, subset_by_index=[n, n + nev - 1], driver="evr")
        return lam
    lam, q = sla.eigh(Hh, subset_by_index=[n, n + nev - 1], driver="evr")
    y = sla.solve_triangular(L.T, q, lower=False)
    Z = shao_q(n) @ y
    J = omega_metric(n)
    jn = np.real(np.einsum("ij,ij->j", Z.conj(), J @ Z))
    Z = Z / np.sqrt(jn)
    return lam, Z[:n], Z[n:]


# ---------------------------------------------------------------- operators
def apply_bse(A, B, X):
    """Y = H X with H of Eq. 1 (formed densely)."""
    return bse_hamiltonian(A, B) @ _c128(X)


def apply_a(A, X):
    """Y = A X (the TDA operator)."""
    return _c128(A) @ _c128(X)


def apply_mplus(A, B, U):
    """M+ U = A U + B conj(U): the real-linear half of H on the conjugation-even
    vectors (X; conj X) (its real matrix is M_r of Eq. 5 with y -> -y)."""
    U = _c128(U)
    return _c128(A) @ U + _c128(B) @ U.conj()


def apply_mminus(A, B, W):
    """M- W = A W - B conj(W); M- M+ has eigenvalues omega^2 (the folded
    operator of Sec. 2.2.1)."""
    W = _c128(W)
    return _c128(A) @ W - _c128(B) @ W.conj()


# ---------------------------------------------------------------- gradients
def hf_gradient_tda(X, g):
    """dL/dA for L(lambda), TDA: G_A = X diag(g) X^H (Hellmann-Feynman,
    d lambda_i = x_i^H dA x_i for unit x_i).  Convention: dL = Re<G, dA>
    with <G, E> = sum conj(G_ij) E_ij."""
    X = _c128(X)
    return (X * np.asarray(g, dtype=np.float64)) @ X.conj().T


def hf_gradient_ph(X, Y, g):
    """dL/dA, dL/dB for L(omega) of the pseudo-Hermitian problem.

    With the left eigenvector Omega z (Eq. 7) and z^H Omega z = 1,
    d omega = z^H Omega dH z = X^H dA X + X^H dB Y + Y^H conj(dB) X + Y^H conj(dA) Y,
    so, with dL = Re<G_A, dA> + Re<G_B, dB>:
        G_A = X diag(g) X^H + conj(Y diag(g) Y^H)
        G_B = X diag(g) Y^H + (X diag(g) Y^H)^T  (complex symmetric)."""
    X = _c128(X)
    Y = _c128(Y)
    g = np.asarray(g, dtype=np.float64)
    ga = (X * g) @ X.conj().T + ((Y * g) @ Y.conj().T).conj()
    xy = (X * g) @ Y.conj().T
    gb = xy + xy.T
    return ga, gb


# ---------------------------------------------------------------- checks
def relative_residuals_ph(A, B, omega, X, Y):
    """||H z - omega z||_2 / (|omega| ||z||_2) per column."""
    Z = np.vstack([_c128(X), _c128(Y)])
    R = apply_bse(A, B, Z) - Z * np.asarray(omega)
    return np.linalg.norm(R, axis=0) / (np.abs(omega) * np.linalg.norm(Z, axis=0))


def relative_residuals_tda(A, lam, X):
    X = _c128(X)
    R = apply_a(A, X) - X * np.asarray(lam)
    return np.linalg.norm(R, axis=0) / (np.abs(lam) * np.linalg.norm(X, axis=0))


def j_rayleigh_quotients(A, B, X, Y):
    """rho = Re(z^H Omega H z) / (z^H Omega z) per column (Eq. 3: Omega H = M)."""
    Z = np.vstack([_c128(X), _c128(Y)])
    n = Z.shape[0] // 2
    J = omega_metric(n)
    HZ = apply_bse(A, B, Z)
    num = np.real(np.einsum("ij,ij->j", Z.conj(), J @ HZ))
    den = np.real(np.einsum("ij,ij->j", Z.conj(), J @ Z))
    return num / den
