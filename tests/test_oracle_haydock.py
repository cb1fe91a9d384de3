"""Pins of the Haydock oracle (oracle/haydock.py) against closed forms,
symmetries, sum rules and the exactness of an N-step Lanczos recurrence.

The response definitions (dense solves) are pinned by the 1x1 / 2x2 block
closed forms; the three-term recurrences are pinned by reaching those
definitions exactly after N steps and by the trace of the tridiagonal
matrix; nothing here compares the oracle with itself."""
import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(2504)


def _herm(n, rng, shift, scale):
    x = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * scale
    return (x + x.conj().T) / 2 + shift * np.eye(n)


def _sym(n, rng, scale):
    x = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * scale
    return (x + x.T) / 2


def _cvec(n, rng):
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


Z = np.array([1.3 + 0.05j, 2.9 + 0.1j, 3.4 + 0.02j, -2.2 + 0.3j, 6.0 + 1.0j])


def test_tda_diagonal_closed_form():
    a = np.array([1.5, 2.0, 2.7, 4.1])
    d = _cvec(4, RNG)
    F = O.response_tda(np.diag(a), d, Z)
    ref = np.array([np.sum(np.abs(d) ** 2 / (z - a)) for z in Z])
    np.testing.assert_allclose(F, ref, rtol=1e-13)


@pytest.mark.parametrize("sign", [-1, 1])
def test_ph_diagonal_blocks_closed_form(sign):
    """Diagonal A and B decouple H into 2x2 blocks [[a, b], [-conj b, -a]]:
    F = sum_i (2 a_i |d_i|^2 + 2 s Re(conj(b_i) d_i^2)) / (z^2 - a_i^2 + |b_i|^2)."""
    a = np.array([1.8, 2.4, 3.0, 3.9, 5.2])
    b = np.array([0.3 + 0.2j, -0.1j, 0.5, 0.2 - 0.4j, 0.0])
    d = _cvec(5, RNG)
    F = O.response_ph(np.diag(a), np.diag(b), d, Z, sign=sign)
    num = 2 * a * np.abs(d) ** 2 + 2 * sign * np.real(np.conj(b) * d ** 2)
    ref = np.array([np.sum(num / (z * z - a ** 2 + np.abs(b) ** 2)) for z in Z])
    np.testing.assert_allclose(F, ref, rtol=1e-12)


def test_ph_b_zero_is_tda_pair():
    A = _herm(7, RNG, 3.0, 0.3)
    d = _cvec(7, RNG)
    F = O.response_ph(A, np.zeros((7, 7)), d, Z)
    ref = O.response_tda(A, d, Z) + O.response_tda(A, d, -Z)
    np.testing.assert_allclose(F, ref, rtol=1e-12)


def test_ph_sign_is_b_flip():
    A = _herm(6, RNG, 3.0, 0.3)
    B = _sym(6, RNG, 0.1)
    d = _cvec(6, RNG)
    np.testing.assert_allclose(O.response_ph(A, B, d, Z, sign=1), O.response_ph(A, -B, d, Z, sign=-1),
                               rtol=1e-12)


@pytest.mark.parametrize("sign", [-1, 1])
def test_ph_positivity_and_sum_rule(sign):
    """-Im F(omega + i eta) > 0 for omega, eta > 0 (M positive definite), and
    z^2 F(z) -> 2 Re(d^H K d) (K = M- for s = -1, M+ for s = +1) as |z| grows."""
    n = 8
    A = _herm(n, RNG, 3.0, 0.3)
    B = _sym(n, RNG, 0.1)
    d = _cvec(n, RNG)
    w = np.linspace(0.5, 6.0, 23) + 0.05j
    assert np.all(O.spectrum_from_response(O.response_ph(A, B, d, w, sign=sign)) > 0)
    K = O.apply_mminus if sign < 0 else O.apply_mplus
    C = 2 * np.real(np.vdot(d, K(A, B, d)))
    z = np.array([1e5j])
    np.testing.assert_allclose((z * z * O.response_ph(A, B, d, z, sign=sign)).real, C, rtol=1e-8)


def test_lanczos_tda_exact_after_n_steps():
    n = 10
    A = _herm(n, RNG, 3.0, 0.4)
    d = _cvec(n, RNG)
    al, be, n2 = O.lanczos_tda(A, d, n)
    assert len(al) == n
    np.testing.assert_allclose(np.sum(al), np.trace(A).real, rtol=1e-12)     # T_N similar to A
    np.testing.assert_allclose(O.haydock_response_tda(A, d, n, Z), O.response_tda(A, d, Z), rtol=1e-9)


@pytest.mark.parametrize("sign", [-1, 1])
def test_lanczos_ph_exact_after_n_steps(sign):
    """The folded operator has each omega^2 twice; the Krylov space of one
    start vector holds one direction per pair, so N steps are exact."""
    n = 10
    A = _herm(n, RNG, 3.0, 0.4)
    B = _sym(n, RNG, 0.15)
    d = _cvec(n, RNG)
    al, be, n2 = O.lanczos_ph(A, B, d, n, sign=sign)
    om = O.ph_full_spectrum(A, B)
    om = np.sort(om.real[om.real > 0])
    np.testing.assert_allclose(np.sum(al), np.sum(om ** 2), rtol=1e-11)
    np.testing.assert_allclose(O.haydock_response_ph(A, B, d, n, Z, sign=sign),
                               O.response_ph(A, B, d, Z, sign=sign), rtol=1e-8)


def test_continued_fraction_two_level():
    """CF of a 2x2 Jacobi matrix equals its (1,1) resolvent entry."""
    a1, a2, b = 1.0, 3.0, 0.7
    T = np.array([[a1, b], [b, a2]])
    z = np.array([0.5 + 0.1j, 2.0 + 0.2j])
    ref = np.array([np.linalg.inv(zz * np.eye(2) - T)[0, 0] for zz in z])
    np.testing.assert_allclose(O.continued_fraction([a1, a2], [b], z), ref, rtol=1e-14)
