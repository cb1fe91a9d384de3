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
