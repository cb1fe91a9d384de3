"""CPU check of the double-FP32 arithmetic the mixed and df64 products use.

Emulated with numpy float32 (round-to-nearest, one IEEE operation per call,
exactly what the __f*_rn intrinsics and the f32x2 lanes do): Dekker's product
(the FMA gives the exact rounding error of fl(a x)), Knuth's TwoSum, and the
(hi, lo) accumulation of a dot product.  The exact reference is rational
arithmetic (fractions.Fraction), so the checks are against the true sums, not
against another floating-point computation."""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    bp = f32(s - a)
    e = f32(f32(a - f32(s - bp)) + f32(b - bp))
    return s, e


def fma32(a, b, c):
    """float32 fused multiply-add: exact product and sum, one rounding."""
    return f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def df_acc(h, l, ah, al, xh, xl):
    """(h, l) += (ah + al)(xh + xl) as the kernels do it (a_lo x_lo dropped)."""
    p = f32(ah * xh)
    e = fma32(ah, xh, -p)
    e = fma32(ah, xl, e)
    e = fma32(al, xh, e)
    t, err = two_sum(h, p)
    return t, f32(l + f32(err + e))


def split32(v):
    hi = f32(v)
    return hi, f32(v - float(hi))


def test_two_sum_is_exact():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        a, b = (f32(v) for v in rng.standard_normal(2) * 10.0 ** rng.integers(-8, 8, 2))
        s, e = two_sum(a, b)
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(a)) + Fraction(float(b))


def test_dekker_error_term_is_exact():
    rng = np.random.default_rng(2)
    for _ in range(2000):
        a, x = (f32(v) for v in rng.standard_normal(2))
        p = f32(a * x)
        e = fma32(a, x, -p)
        assert Fraction(float(p)) + Fraction(float(e)) == Fraction(float(a)) * Fraction(float(x))


@pytest.mark.parametrize("n", [8, 128, 1024])
def test_double_fp32_dot_product_reaches_2_pow_minus_44(n):
    """A length-n dot product of split FP64 operands accumulated in (hi, lo)
    FP32 pairs: the error is a few 2^-48 per term of the sum of |terms|,
    the FP64-class accuracy the mixed path relies on (plain FP32: ~2^-24)."""
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n)
    x = rng.standard_normal(n)
    h, l = f32(0.0), f32(0.0)
    for ai, xi in zip(a, x):
        ah, al = split32(ai)
        xh, xl = split32(xi)
        h, l = df_acc(h, l, ah, al, xh, xl)
    got = Fraction(float(h)) + Fraction(float(l))
    exact = sum(Fraction(float(ai)) * Fraction(float(xi)) for ai, xi in zip(a, x))
    scale = sum(abs(Fraction(float(ai)) * Fraction(float(xi))) for ai, xi in zip(a, x))
    assert abs(got - exact) <= scale * Fraction(2) ** -44
    plain = f32(0.0)
    for ai, xi in zip(a, x):
        plain = f32(plain + f32(f32(ai) * f32(xi)))
    # and it is far better than plain FP32 accumulation
    assert abs(got - exact) * 1000 < abs(Fraction(float(plain)) - exact) + scale * Fraction(2) ** -60


def test_exact_complex64_values_give_exact_u_v():
    """U = A + sB, V = A - sB formed by TwoSum from exact FP32 A and B are exact
    as (hi, lo) pairs (what the mixed path's kernel relies on)."""
    rng = np.random.default_rng(5)
    for _ in range(2000):
        a, b = (f32(v) for v in rng.standard_normal(2) * 10.0 ** rng.integers(-3, 3, 2))
        for s in (1.0, -1.0):
            hi, lo = two_sum(a, f32(s * b))
            assert Fraction(float(hi)) + Fraction(float(lo)) == Fraction(float(a)) + Fraction(s) * Fraction(float(b))


def tf32_rna(v):
    """Round a float32 to TF32 (10 explicit mantissa bits), nearest, ties away
    from zero: the cvt.rna.tf32.f32 the adjoint's panel kernel uses."""
    b = np.float32(v).view(np.uint32)
    b = (b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    return b.view(np.float32)


def test_three_tf32_products_reach_fp32_class_accuracy():
    """3xTF32 (hi*hi + hi*lo + lo*hi, FP32 accumulation) for the adjoint's
    rank-2k update: the per-product error stays at the FP32 level (2^-21),
    where one TF32 product is at 2^-10."""
    rng = np.random.default_rng(9)
    a = rng.standard_normal(4096).astype(np.float32)
    b = rng.standard_normal(4096).astype(np.float32)
    ah = tf32_rna(a); al = (a - ah).astype(np.float32)
    bh = tf32_rna(b); bl = (b - bh).astype(np.float32)
    # the tensor core reads the lo parts as TF32 too: model the worst case, truncation
    trunc = lambda v: (v.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
    alt, blt = trunc(al), trunc(bl)
    exact = a.astype(np.float64) * b.astype(np.float64)
    three = (ah.astype(np.float64) * bh + ah.astype(np.float64) * blt + alt.astype(np.float64) * bh)
    one = ah.astype(np.float64) * bh
    rel3 = np.max(np.abs(three - exact) / np.abs(exact))
    rel1 = np.max(np.abs(one - exact) / np.abs(exact))
    assert rel3 < 2.0 ** -20
    assert rel1 > 2.0 ** -12
    # the split is exact: hi + lo == a, and lo fits in TF32 up to its own rounding
    assert np.array_equal((ah + al).astype(np.float32), a)
