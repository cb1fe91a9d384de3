"""GPU parity of the Hellmann-Feynman adjoint (bse_backward) against the
oracle's gradient from its own eigenvectors, and of the torch.autograd
wrapper against central finite differences of the GPU eigenvalues."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import problem, rand_block, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_backward_ph_fp64_matches_oracle():
    from paper_2504_10096_gb300 import bse
    n, nev = 257, 6
    A, B = problem(n, "c128", seed=31)
    s = bse.Solver(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    vals, _, _ = s.solve(nev, tol=1e-13)
    g = np.random.default_rng(1).uniform(0.1, 1.0, nev)
    dA, dB = s.backward(g)
    om, X, Y = O.ph_lowest(A, B, nev)
    GA, GB = O.hf_gradient_ph(X, Y, g)
    assert rel(dA.cpu().numpy(), GA) < 1e-8
    assert rel(dB.cpu().numpy(), GB) < 1e-8
    s.close()


def test_backward_tda_fp64_matches_oracle():
    from paper_2504_10096_gb300 import bse
    n, nev = 300, 5
    A, _ = problem(n, "c128", form="tda", seed=33)
    s = bse.Solver(torch.from_numpy(A).cuda())
    s.solve(nev, tol=1e-13)
    g = np.linspace(0.2, 1.0, nev)
    dA, dB = s.backward(g)
    assert dB is None
    lam, X = O.tda_lowest(A, nev)
    assert rel(dA.cpu().numpy(), O.hf_gradient_tda(X, g)) < 1e-8
    s.close()


def test_backward_c64_error_stated():
    from paper_2504_10096_gb300 import bse
    n, nev = 300, 6
    A, B = problem(n, "c64", seed=35)
    s = bse.Solver(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), mixed=True)
    s.solve(nev, tol=1e-6)
    g = np.ones(nev)
    dA, dB = s.backward(g)
    om, X, Y = O.ph_lowest(A.astype(np.complex128), B.astype(np.complex128), nev)
    GA, GB = O.hf_gradient_ph(X, Y, g)
    assert rel(dA.cpu().numpy(), GA) < 1e-3
    assert rel(dB.cpu().numpy(), GB) < 1e-3
    s.close()


@pytest.mark.parametrize("form,n,nev", [("ph", 300, 6), ("tda", 333, 5), ("ph", 1000, 40), ("ph", 3000, 8)])
def test_backward_tensor_cores_match_cuda_cores(form, n, nev):
    """tcgen05 3xTF32 rank-2k update against the FP32 CUDA-core kernel on the
    same eigenvectors: ragged tiles, several K chunks, more tiles than SMs."""
    from paper_2504_10096_gb300 import bse
    A, B = problem(n, "c64", form=form, seed=41 + n)
    s = bse.Solver(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda() if form == "ph" else None, mixed=True)
    s.solve(nev, tol=1e-6)
    g = np.random.default_rng(5).uniform(-1.0, 1.0, nev)
    dA1, dB1 = s.backward(g, impl=bse.BSE_IMPL_CUDA_CORES)
    dA2, dB2 = s.backward(g, impl=bse.BSE_IMPL_TENSOR_CORES)
    a1, a2 = dA1.cpu().numpy(), dA2.cpu().numpy()
    assert rel(a2, a1) < 2e-5
    assert np.array_equal(a2, a2.conj().T)          # Hermitian by construction (mirror writes)
    if form == "ph":
        b1, b2 = dB1.cpu().numpy(), dB2.cpu().numpy()
        assert rel(b2, b1) < 2e-5
        assert np.array_equal(b2, b2.T)
    s.close()


@pytest.mark.parametrize("form,n,nev", [("ph", 300, 6), ("ph", 1000, 40), ("tda", 333, 5)])
def test_tensor_core_adjoint_elementwise_on_own_vectors(form, n, nev):
    """k_adjoint_tc against oracle.hf_gradient_ph / hf_gradient_tda evaluated on
    the GPU's own returned eigenvectors, entry by entry: this isolates the
    tcgen05 kernel (3xTF32 products, FP32 accumulation in tensor memory,
    complex64 output) from the eigenvector error of the solve.  Bound per
    entry: (8 2^-21 + 3 K 2^-23) (sum_k |g_k| (|X_ik||X_jk| + |Y_ik||Y_jk|)) for
    G_A, the same with |X_ik||Y_jk| + |Y_ik||X_jk| for G_B: three TF32 hi/lo
    products per term (the dropped lo x lo and the lo parts' own rounding, a few
    2^-22), K = 2 nev (PH) or nev (TDA) rank-one terms, each three MMAs,
    accumulated in FP32."""
    from paper_2504_10096_gb300 import bse
    A, B = problem(n, "c64", form=form, seed=51 + n)
    s = bse.Solver(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda() if form == "ph" else None, mixed=True)
    _, vecs, _ = s.solve(nev, tol=1e-8)
    g = np.random.default_rng(7).uniform(-1.0, 1.0, nev)
    dA, dB = s.backward(g, impl=bse.BSE_IMPL_TENSOR_CORES)
    Z = vecs.cpu().numpy().astype(np.complex128)
    ag = np.abs(g)
    if form == "ph":
        X, Y = Z[:n], Z[n:]
        GA, GB = O.hf_gradient_ph(X, Y, g)
        aX, aY = np.abs(X), np.abs(Y)
        bA = (aX * ag) @ aX.T + (aY * ag) @ aY.T
        bB = (aX * ag) @ aY.T + ((aX * ag) @ aY.T).T
        pairs = ((dA, GA, bA), (dB, GB, bB))
    else:
        GA = O.hf_gradient_tda(Z, g)
        aX = np.abs(Z)
        pairs = ((dA, GA, (aX * ag) @ aX.T),)
    K = 2 * nev if form == "ph" else nev
    c = 8 * 2.0 ** -21 + 3 * K * 2.0 ** -23
    for got, ref, bnd in pairs:
        err = np.abs(got.cpu().numpy().astype(np.complex128) - ref)
        worst = float(np.max(err / (c * bnd + 1e-30)))
        assert worst <= 1.0, worst
    s.close()


def test_autograd_against_finite_differences():
    from paper_2504_10096_gb300 import bse
    n, nev = 140, 4
    A, B = problem(n, "c128", seed=37)
    At = torch.from_numpy(A).cuda().requires_grad_(True)
    Bt = torch.from_numpy(B).cuda().requires_grad_(True)
    w = torch.tensor([0.3, 0.9, 0.5, 0.7], dtype=torch.float64, device="cuda")
    lam = bse.bse_eigenvalues(At, Bt, nev, tol=1e-13)
    (lam * w).sum().backward()
    GA, GB = At.grad.cpu().numpy(), Bt.grad.cpu().numpy()

    def loss(a, b):
        s = bse.Solver(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
        v, _, _ = s.solve(nev, tol=1e-13, vectors=False)
        s.close()
        return float(np.dot(w.cpu().numpy(), v))

    h = 1e-5
    rng = np.random.default_rng(3)
    for _ in range(4):
        i, j = (int(x) for x in rng.integers(0, n, 2))
        if i == j:
            continue
        E = np.zeros((n, n), complex)
        E[i, j] = E[j, i] = 1.0
        fd = (loss(A + h * E, B) - loss(A - h * E, B)) / (2 * h)
        assert abs(fd - 2 * GA[i, j].real) < 1e-6
        E2 = np.zeros((n, n), complex)
        E2[i, j] = E2[j, i] = 1j
        fd = (loss(A, B + h * E2) - loss(A, B - h * E2)) / (2 * h)
        assert abs(fd - 2 * GB[i, j].imag) < 1e-6
