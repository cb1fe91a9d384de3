"""Parity at the full workload sizes, in the launch configuration bench.py
times: config 1 (pseudo-Hermitian, N = 10000, complex128, lowest 100, FP64)
against eigenvalues the oracle stored (tests/golden/make_golden.py), plus the
properties that hold at any size (residuals, Omega-normalisation, sampled
rows of H z recomputed on the host)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_config1_ph_n10000_fp64():
    from paper_2504_10096_gb300 import bse
    from synthetic import CONFIGS, make_problem_torch
    spec = CONFIGS[1]
    p = make_problem_torch(spec, device="cuda")
    A, B = p["A"], p["B"]
    s = bse.Solver(A, B)
    vals, vecs, nconv = s.solve(spec.nev, tol=1e-12)
    gold = np.loadtxt(os.path.join(GOLD, "config1_omega.txt"))
    assert nconv == spec.nev
    np.testing.assert_allclose(vals, gold, rtol=1e-10, atol=0)
    assert s.stats()["max_residual"] < 1e-11
    # sampled rows of H z recomputed on the host from the stored blocks
    n = spec.n
    rows = np.random.default_rng(0).choice(n, 16, replace=False)
    cols = [0, 37, 99]
    Z = vecs[:, cols].cpu().numpy()
    Ar = A[rows].cpu().numpy()
    Br = B[rows].cpu().numpy()
    X, Y = Z[:n], Z[n:]
    hz1 = Ar @ X + Br @ Y                       # first block row of H z
    np.testing.assert_allclose(hz1, X[rows] * vals[cols], rtol=0, atol=1e-10 * np.abs(X).max())
    jn = np.sum(np.abs(X) ** 2, 0) - np.sum(np.abs(Y) ** 2, 0)
    np.testing.assert_allclose(jn, 1.0, atol=1e-10)
    s.close()


def test_config2_batch_of_64_uneven():
    """Workload config 2: 64 pseudo-Hermitian problems, N_i ~ U{500..6000},
    complex64, lowest 16 each, solved in lock-step launches; eigenvalues
    against the per-problem FP64 oracle (stored), 1e-6 relative after the
    FP64 Rayleigh-quotient refinement."""
    from paper_2504_10096_gb300 import bse
    from synthetic import batched_specs, make_problem_torch
    specs = batched_specs()
    As, Bs = [], []
    for sp in specs:
        p = make_problem_torch(sp, device="cuda")
        As.append(p["A"])
        Bs.append(p["B"])
    bs = bse.BatchedSolver(As, Bs)
    del As, Bs
    nev = specs[0].nev
    vals, _, nconv = bs.solve(nev, tol=1e-6)
    gold = np.loadtxt(os.path.join(GOLD, "config2_omega.txt")).reshape(len(specs), nev)
    assert np.all(nconv == nev)
    np.testing.assert_allclose(vals, gold, rtol=1e-6, atol=0)
    assert bs.stats()["max_residual"] < 1e-4
    bs.close()
