"""Helpers shared by the GPU parity tests (inputs only; no solver arithmetic)."""
import numpy as np

from synthetic import BSEProblemSpec, make_problem


def problem(n, dtype="c128", form="ph", seed=3, n_g=None):
    spec = BSEProblemSpec(n=n, n_g=n_g or max(8, min(200, n // 4)), seed=seed, form=form, dtype=dtype)
    p = make_problem(spec)
    return p["A"], p["B"]


def rand_block(n, k, dtype, seed=0):
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))) / np.sqrt(2)
    return x.astype(np.complex64 if dtype == "c64" else np.complex128)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def omega_metric_apply(Z):
    n = Z.shape[0] // 2
    out = Z.copy()
    out[n:] *= -1
    return out


# unit roundoff of the storage precision of the product tests
UNIT = {"c128": 2.0 ** -53, "c64": 2.0 ** -24}


def product_bound(A, B, X, op):
    """Element-wise magnitude |M| |X| that bounds the rounding of Y = M X
    (M = A, M+/M- with both blocks, or H of Eq. 1 for op "h"), in FP64."""
    aA = np.abs(np.asarray(A, dtype=np.complex128))
    aX = np.abs(np.asarray(X, dtype=np.complex128))
    if op == "a":
        return aA @ aX
    aB = np.abs(np.asarray(B, dtype=np.complex128))
    if op in ("mplus", "mminus"):
        return aA @ aX + aB @ aX
    n = aA.shape[0]
    x1, x2 = aX[:n], aX[n:]
    return np.vstack([aA @ x1 + aB @ x2, aB @ x1 + aA @ x2])


def assert_elementwise(Y, Yref, bound, u, c, what=""):
    """|Y - Yref| <= c u bound element by element (bound from product_bound)."""
    err = np.abs(np.asarray(Y, dtype=np.complex128) - np.asarray(Yref, dtype=np.complex128))
    lim = c * u * np.asarray(bound) + 1e-300
    worst = float(np.max(err / lim))
    assert worst <= 1.0, f"{what}: element error reaches {worst:.3g} x the bound {c} u |M||x|"
    return worst
