"""GPU parity of the Lanczos-Haydock spectrum (bse_haydock) against the
oracle: the dense resolvent definition once the continued fraction has
converged (m = 2N steps), and the oracle's own three-term recurrence for the
leading coefficients (before loss of orthogonality separates the two
rounding histories)."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import problem, rand_block

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

OMEGA = np.linspace(0.5, 12.0, 47)
ETA = 0.1


def _solver(A, B=None, **kw):
    from paper_2504_10096_gb300 import bse
    return bse.Solver(torch.from_numpy(A).cuda(), None if B is None else torch.from_numpy(B).cuda(), **kw)


def _maxrel(F, G):
    return float(np.max(np.abs(F - G)) / np.max(np.abs(G)))


def test_haydock_tda_matches_dense_resolvent():
    n = 333
    A, _ = problem(n, "c128", form="tda", seed=61)
    d = rand_block(n, 1, "c128", seed=1)[:, 0]
    s = _solver(A)
    spec, F, coefs, steps = s.haydock(d, 2 * n, OMEGA, ETA)
    Fo = O.response_tda(A, d, OMEGA + 1j * ETA)
    assert steps == 2 * n
    assert _maxrel(F, Fo) < 1e-9
    np.testing.assert_allclose(spec, O.spectrum_from_response(Fo), rtol=0, atol=1e-9 * np.max(np.abs(Fo)))
    al, be, n2 = O.lanczos_tda(A, d, 20)
    np.testing.assert_allclose(coefs["alpha"][:20], al, rtol=1e-11)
    np.testing.assert_allclose(coefs["beta"][:19], be, rtol=1e-10)
    np.testing.assert_allclose(coefs["norm2"], n2, rtol=1e-13)
    s.close()


@pytest.mark.parametrize("sign", [-1, 1])
def test_haydock_ph_matches_dense_resolvent(sign):
    n = 300
    A, B = problem(n, "c128", seed=63)
    d = rand_block(n, 1, "c128", seed=2)[:, 0]
    s = _solver(A, B)
    spec, F, coefs, steps = s.haydock(d, 2 * n, OMEGA, ETA, sign=sign)
    Fo = O.response_ph(A, B, d, OMEGA + 1j * ETA, sign=sign)
    assert _maxrel(F, Fo) < 1e-9
    assert np.all(spec[OMEGA > 0] > -1e-9 * np.max(np.abs(Fo)))
    al, be, n2 = O.lanczos_ph(A, B, d, 20, sign=sign)
    np.testing.assert_allclose(coefs["alpha"][:20], al, rtol=1e-11)
    np.testing.assert_allclose(coefs["beta"][:19], be, rtol=1e-10)
    np.testing.assert_allclose(coefs["norm2"], n2, rtol=1e-12)
    s.close()


@pytest.mark.parametrize("mode", ["c64", "mixed", "c128_df"])
def test_haydock_reduced_precision_paths(mode):
    """complex64 storage with FP32 vectors (c64), with FP64 vectors and
    double-FP32 products (mixed), complex128 with double-FP32 products."""
    n = 260
    dt = "c128" if mode == "c128_df" else "c64"
    A, B = problem(n, dt, seed=65)
    d = rand_block(n, 1, "c128", seed=3)[:, 0]
    s = _solver(A, B, mixed=(mode == "mixed"), df=(mode == "c128_df"))
    _, F, _, _ = s.haydock(d, 2 * n, OMEGA, ETA)
    Fo = O.response_ph(A.astype(np.complex128), B.astype(np.complex128), d, OMEGA + 1j * ETA)
    assert _maxrel(F, Fo) < (2e-4 if mode == "c64" else 1e-9)
    s.close()


def test_haydock_invariant_subspace_ends_the_fraction():
    """d spanning three eigenvectors of a diagonal A: the Krylov space is
    three-dimensional, the recurrence stops after three steps and the
    fraction is exact."""
    n = 200
    a = np.linspace(1.5, 9.0, n)
    A = np.diag(a).astype(np.complex128)
    d = np.zeros(n, np.complex128)
    d[[3, 50, 120]] = [1.0, 0.5j, -0.25]
    s = _solver(A)
    spec, F, coefs, steps = s.haydock(d, 50, OMEGA, ETA)
    assert steps == 3
    ref = np.array([np.sum(np.abs(d) ** 2 / (z - a)) for z in OMEGA + 1j * ETA])
    assert _maxrel(F, ref) < 1e-12
    s.close()


def test_haydock_invalid_arguments():
    from paper_2504_10096_gb300 import bse
    n = 140
    A, B = problem(n, "c128", seed=67)
    s = _solver(A, B)
    d = torch.from_numpy(rand_block(n, 1, "c128", seed=4)[:, 0]).cuda()
    for m, sign, eta in [(0, -1, 0.1), (10, 0, 0.1), (10, -1, 0.0), (10, -1, -1.0)]:
        rc, *_ = bse.bse_haydock(s.h, d.data_ptr(), bse.BSE_DEVICE, m, sign, OMEGA, eta)
        assert rc == bse.BSE_EINVAL
    rc, *_ = bse.bse_haydock(s.h, torch.zeros(n, dtype=torch.complex128, device="cuda").data_ptr(),
                             bse.BSE_DEVICE, 10, -1, OMEGA, 0.1)
    assert rc == bse.BSE_ENOTPD
    s.close()
