"""FP64 oracle for the Lanczos-Haydock absorption spectrum.

TEST INFRASTRUCTURE ONLY (same rule as oracle/dense.py): imported by tests/,
__graft_entry__.smoke() and bench.py's CPU legs, never by the product path.

Sec. 2.2 of the paper names the second iterative route of the BSE code it
studies: a Lanczos iteration whose coefficients give the optical absorption
spectrum through quadrature / continued fractions, without eigenvectors
(the "Haydock" solver that is fastest in the size-scaling study of Sec. 3).
The paper prints no formula for it, so the quantities here are this build's
readings, stated once:

* TDA: the response F(z) = d^H (z - A)^{-1} d for a dipole vector d and
  complex frequency z = omega + i eta; spectrum S(omega) = -Im F / pi.
* PH: F(z) = D^H Omega (z - H)^{-1} D with H of Eq. 1 and
  D = (d; s conj(d)), s = -1 or +1.  By the Omega-self-adjointness of H
  (Eq. 7 pairs), F(z) = sum over positive omega_i of
  2 omega_i |z_i^H Omega D|^2 / (z^2 - omega_i^2): a function of z^2.

The plain definitions (dense solves) are `response_tda` / `response_ph`.
The method the GPU runs is a three-term Lanczos recurrence without
re-orthogonalisation whose continued fraction approximates F:

* TDA: Lanczos on A from q1 = d / |d|, F_m(z) = |d|^2 CF_m(z).
* PH, s = -1: Lanczos on the folded operator T~ = M+ M- (M+ u = A u + B conj(u),
  M- w = A w - B conj(w)), self-adjoint in <x, y>_- = Re(x^H M- y), from d;
  F(z) = 2 <d, d>_- CF(z^2).  For s = +1 the roles of M+ and M- swap
  (T = M- M+ in <x, y>_+ = Re(x^H M+ y)), which is the same as s = -1
  with B replaced by -B.

CF_m(zeta) = 1 / (zeta - a_1 - b_1^2 / (zeta - a_2 - ... - b_{m-1}^2 / (zeta - a_m))).
With m equal to the dimension of the Krylov space (N in exact arithmetic)
the continued fraction is exact; the pins in tests/test_oracle_haydock.py
check that against the dense definitions.
"""
from __future__ import annotations

import numpy as np

from .dense import apply_mminus, apply_mplus, bse_hamiltonian, omega_metric

__all__ = [
    "response_tda",
    "response_ph",
    "spectrum_from_response",
    "lanczos_tda",
    "lanczos_ph",
    "continued_fraction",
    "haydock_response_tda",
    "haydock_response_ph",
]


def response_tda(A, d, z):
    """F(z) = d^H (z I - A)^{-1} d, one dense solve per frequency (definition)."""
    A = np.asarray(A, dtype=np.complex128)
    d = np.asarray(d, dtype=np.complex128)
    n = A.shape[0]
    out = np.empty(len(np.atleast_1d(z)), dtype=np.complex128)
    for k, zk in enumerate(np.atleast_1d(z)):
        out[k] = np.vdot(d, np.linalg.solve(zk * np.eye(n) - A, d))
    return out


def response_ph(A, B, d, z, sign=-1):
    """F(z) = D^H Omega (z I - H)^{-1} D, D = (d; sign conj(d)) (definition)."""
    H = bse_hamiltonian(np.asarray(A, np.complex128), np.asarray(B, np.complex128))
    d = np.asarray(d, dtype=np.complex128)
    D = np.concatenate([d, sign * d.conj()])
    Om = omega_metric(d.shape[0])
    n2 = H.shape[0]
    out = np.empty(len(np.atleast_1d(z)), dtype=np.complex128)
    for k, zk in enumerate(np.atleast_1d(z)):
        out[k] = np.vdot(D, Om @ np.linalg.solve(zk * np.eye(n2) - H, D))
    return out


def spectrum_from_response(F):
    """Absorption S = -Im F / pi."""
    return -np.imag(F) / np.pi


def continued_fraction(alpha, beta, zeta):
    """CF_m(zeta) for Lanczos coefficients alpha[0..m-1], beta[0..m-2]
    (beta[j] couples vectors j and j+1), evaluated from the bottom up."""
    alpha = np.asarray(alpha, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    zeta = np.asarray(zeta, dtype=np.complex128)
    m = len(alpha)
    t = np.zeros_like(zeta)
    for j in range(m - 1, -1, -1):
        tail = beta[j] ** 2 * t if j < m - 1 else 0.0
        t = 1.0 / (zeta - alpha[j] - tail)
    return t


def lanczos_tda(A, d, m):
    """Three-term Hermitian Lanczos on A from d / |d| (no re-orthogonalisation).

    Returns (alpha, beta, norm2) with norm2 = |d|^2; stops early (shorter
    arrays) when beta_j^2 <= 1e-28 (|alpha_j| + beta_{j-1})^2, i.e. when the
    Krylov space is invariant to rounding."""
    A = np.asarray(A, dtype=np.complex128)
    d = np.asarray(d, dtype=np.complex128)
    norm2 = float(np.real(np.vdot(d, d)))
    q = d / np.sqrt(norm2)
    q_prev = np.zeros_like(q)
    b_prev = 0.0
    alpha, beta = [], []
    for j in range(m):
        w = A @ q
        a = float(np.real(np.vdot(q, w)))
        alpha.append(a)
        if j == m - 1:
            break
        r = w - a * q - b_prev * q_prev
        b2 = float(np.real(np.vdot(r, r)))
        if not b2 > 1e-28 * (abs(a) + b_prev) ** 2:     # invariant Krylov space: the fraction ends
            break
        b = np.sqrt(b2)
        beta.append(b)
        q_prev, q, b_prev = q, r / b, b
    return np.array(alpha), np.array(beta), norm2


def lanczos_ph(A, B, d, m, sign=-1):
    """Three-term Lanczos on the folded operator of the PH response.

    sign = -1: T~ = M+ M- in <x, y>_- = Re(x^H M- y); sign = +1: T = M- M+ in
    <x, y>_+ = Re(x^H M+ y).  Each step applies the inner-product operator
    K (M- or M+) to the current vector and then the other half to the result:
        p_j = K q_j, w = K' p_j, alpha_j = Re(p_j^H w),
        r = w - alpha_j q_j - beta_{j-1} q_{j-1}, beta_j^2 = Re(r^H K r).
    Returns (alpha, beta, norm2) with norm2 = <d, d>_K."""
    A = np.asarray(A, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    d = np.asarray(d, dtype=np.complex128)
    if sign < 0:
        K = lambda x: apply_mminus(A, B, x)
        Kp = lambda x: apply_mplus(A, B, x)
    else:
        K = lambda x: apply_mplus(A, B, x)
        Kp = lambda x: apply_mminus(A, B, x)
    p = K(d)
    norm2 = float(np.real(np.vdot(d, p)))
    s = np.sqrt(norm2)
    q, p = d / s, p / s
    q_prev = np.zeros_like(q)
    b_prev = 0.0
    alpha, beta = [], []
    for j in range(m):
        w = Kp(p)
        a = float(np.real(np.vdot(p, w)))
        alpha.append(a)
        if j == m - 1:
            break
        r = w - a * q - b_prev * q_prev
        pr = K(r)
        b2 = float(np.real(np.vdot(r, pr)))
        if not b2 > 1e-28 * (abs(a) + b_prev) ** 2:     # invariant Krylov space: the fraction ends
            break
        b = np.sqrt(b2)
        beta.append(b)
        q_prev, q, p, b_prev = q, r / b, pr / b, b
    return np.array(alpha), np.array(beta), norm2


def haydock_response_tda(A, d, m, z):
    """F_m(z) = |d|^2 CF_m(z) from lanczos_tda."""
    al, be, n2 = lanczos_tda(A, d, m)
    return n2 * continued_fraction(al, be[: len(al) - 1], z)


def haydock_response_ph(A, B, d, m, z, sign=-1):
    """F_m(z) = 2 <d, d>_K CF_m(z^2) from lanczos_ph."""
    al, be, n2 = lanczos_ph(A, B, d, m, sign)
    z = np.asarray(z, dtype=np.complex128)
    return 2.0 * n2 * continued_fraction(al, be[: len(al) - 1], z * z)
