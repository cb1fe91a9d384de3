"""CPU checks of the algebra the three structured Lanczos variants rest on (Sec. 2.2.1 names
the variants; these are the facts of the readings, checked on small dense problems in FP64 with
numpy, independently of the GPU code and of the oracle's arithmetic):

* the twins: Krylov vectors u of the folded operator T = M- M+ started from one vector keep
  Im(u^H u') = 0 and Im((M+ u)^H (M+ u')) = 0, which makes the twin spaces i M+ K and i K
  orthogonal to the Krylov space in the M+ / M- inner products;
* the Gruning recurrence (Lanczos of H in the M inner product, even and odd tops) run to the
  full dimension gives a zero-diagonal projection whose positive eigenvalues are the omega of H;
* a kept Ritz pair rotated to (u ~ +- w ~)/sqrt 2 turns the pair block [[0, s], [s, 0]] with the
  hub coupling rho into the leaves +-s with couplings +-rho/sqrt 2 (same spectrum);
* the projected BSE matrix [[A_k, B_k], [-B_k, -A_k]] with A_k = (T + I)/2, B_k = (I - T)/2 has
  the eigenvalues +-sqrt(eig T), its M_r (Eq. 5) is diag(I, T), and an eigenvector (a; b)
  gives the folded Ritz coefficients a + b."""
import numpy as np

import oracle as O
from tests.gpu_common import problem


def _ops(A, B):
    Mp = lambda u: A @ u + B @ u.conj()
    Mm = lambda u: A @ u - B @ u.conj()
    return Mp, Mm


def test_twin_orthogonality_of_krylov_vectors():
    A, B = problem(120, "c128", seed=5)
    Mp, Mm = _ops(A, B)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(120) + 1j * rng.standard_normal(120)
    K = [u / np.linalg.norm(u)]
    for _ in range(5):
        v = Mm(Mp(K[-1]))
        K.append(v / np.linalg.norm(v))
    K = np.array(K).T
    P = np.array([Mp(x) for x in K.T]).T
    P /= np.linalg.norm(P, axis=0)
    assert np.abs(np.imag(K.conj().T @ K)).max() < 1e-12
    assert np.abs(np.imag(P.conj().T @ P)).max() < 1e-12
    # the mixed products are not real in general (the fact is specific to the pairs above)
    assert np.abs(np.imag(P.conj().T @ K)).max() > 1e-6


def _gruning_full(A, B, m, seed=2):
    """Lanczos of H in the M inner product on the tops (even u with p = M+ u, odd w with
    z = M- w), full reorthogonalisation with the twin projections, m steps."""
    N = A.shape[0]
    Mp, Mm = _ops(A, B)
    U = np.zeros((N, m + 1), complex); P = np.zeros_like(U)
    W = np.zeros((N, m), complex); Z = np.zeros_like(W)
    al = np.zeros(m); be = np.zeros(m)

    def cgs(x, Xm, Ym, nm, Xt, Yt, nt):
        for _ in range(2):
            x = x - Xm[:, :nm] @ np.real(Ym[:, :nm].conj().T @ x) - 1j * (Xt[:, :nt] @ np.imag(Yt[:, :nt].conj().T @ x))
        return x

    rng = np.random.default_rng(seed)
    s = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    p = Mp(s)
    b = np.sqrt(np.real(np.vdot(s, p)))
    U[:, 0], P[:, 0] = s / b, p / b
    for j in range(m):
        r = cgs(P[:, j].copy(), W, Z, j, U, P, j + 1)
        z = Mm(r)
        al[j] = np.sqrt(np.real(np.vdot(r, z)))
        W[:, j], Z[:, j] = r / al[j], z / al[j]
        s = cgs(Z[:, j].copy(), U, P, j + 1, W, Z, j + 1)
        p = Mp(s)
        be[j] = np.sqrt(max(np.real(np.vdot(s, p)), 0.0))
        if be[j] > 0:
            U[:, j + 1], P[:, j + 1] = s / be[j], p / be[j]
    return al, be, U, W


def test_gruning_projection_has_zero_diagonal_and_the_omegas():
    n = 24
    A, B = problem(n, "c128", seed=11)
    om = O.ph_lowest(A, B, n)[0]
    al, be, U, W = _gruning_full(A, B, n)
    # tridiagonal of order 2n: zero diagonal, couplings alpha_0, beta_0, alpha_1, ...
    e = np.empty(2 * n - 1)
    e[0::2] = al
    e[1::2] = be[:-1]
    T = np.diag(e, 1) + np.diag(e, -1)
    ev = np.linalg.eigvalsh(T)
    np.testing.assert_allclose(ev[n:], om, rtol=1e-10)
    np.testing.assert_allclose(ev[:n], -om[::-1], rtol=1e-10)
    # the even and odd bases are orthonormal in their inner products
    Mp, Mm = _ops(A, B)
    G = np.real(U[:, :n].conj().T @ np.array([Mp(x) for x in U[:, :n].T]).T)
    np.testing.assert_allclose(G, np.eye(n), atol=1e-10)
    G = np.real(W.conj().T @ np.array([Mm(x) for x in W.T]).T)
    np.testing.assert_allclose(G, np.eye(n), atol=1e-10)


def test_rotated_kept_pairs_keep_the_spectrum():
    rng = np.random.default_rng(3)
    h, q = 4, 6
    sig = np.sort(rng.uniform(0.5, 3.0, h))
    rho = rng.standard_normal(h)
    tail = rng.uniform(0.5, 2.0, 2 * q - 1)
    # unrotated: nodes (c_i, r_i) for the kept pairs, hub c_l, then the path r_l, c_{l+1}, ...
    n = 2 * h + 2 * q
    T = np.zeros((n, n))
    for i in range(h):
        T[2 * i, 2 * i + 1] = T[2 * i + 1, 2 * i] = sig[i]          # c_i -- r_i
        T[2 * i + 1, 2 * h] = T[2 * h, 2 * i + 1] = rho[i]          # r_i -- hub
    for t in range(2 * q - 1):
        T[2 * h + t, 2 * h + t + 1] = T[2 * h + t + 1, 2 * h + t] = tail[t]
    # rotated: leaves +sig (coupling rho/sqrt2), -sig (coupling -rho/sqrt2), then hub and path
    R = np.zeros((n, n))
    d = np.concatenate([sig, -sig])
    bb = np.concatenate([rho, -rho]) / np.sqrt(2.0)
    R[np.arange(2 * h), np.arange(2 * h)] = d
    R[2 * h, :2 * h] = bb
    R[:2 * h, 2 * h] = bb
    for t in range(2 * q - 1):
        R[2 * h + t, 2 * h + t + 1] = R[2 * h + t + 1, 2 * h + t] = tail[t]
    np.testing.assert_allclose(np.linalg.eigvalsh(R), np.linalg.eigvalsh(T), rtol=1e-12, atol=1e-12)
    ev = np.linalg.eigvalsh(T)
    np.testing.assert_allclose(ev, -ev[::-1], atol=1e-12)             # spectrum +-sigma


def test_projected_bse_matrix():
    rng = np.random.default_rng(4)
    n = 10
    X = rng.standard_normal((n, n))
    T = X @ X.T + 0.5 * np.eye(n)
    Ak, Bk = (T + np.eye(n)) / 2, (np.eye(n) - T) / 2
    H = np.block([[Ak, Bk], [-Bk, -Ak]])
    w, V = np.linalg.eig(H)
    order = np.argsort(w.real)
    w, V = w[order].real, V[:, order]
    th = np.linalg.eigvalsh(T)
    np.testing.assert_allclose(w[n:], np.sqrt(th), rtol=1e-10)
    np.testing.assert_allclose(w[:n], -np.sqrt(th)[::-1], rtol=1e-10)
    # M_r of Eq. 5 for real blocks: [[A + B, 0], [0, A - B]] = diag(I, T)
    Mr = np.block([[Ak + Bk, np.zeros((n, n))], [np.zeros((n, n)), Ak - Bk]])
    np.testing.assert_allclose(Mr, np.block([[np.eye(n), np.zeros((n, n))], [np.zeros((n, n)), T]]), atol=1e-14)
    for k in range(n, 2 * n):
        c = V[:n, k] + V[n:, k]
        c = c / np.linalg.norm(c)
        np.testing.assert_allclose(T @ c, w[k] ** 2 * c, atol=1e-10 * np.linalg.norm(T))
