"""GPU parity of the batched solve (uneven N, one launch sequence for all
problems) against the per-problem dense oracle."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("dtype,tol,rtol", [("c128", 1e-12, 1e-10), ("c64", 1e-6, 1e-6)])
def test_batched_uneven(dtype, tol, rtol):
    """complex64 runs on the mixed path (FP64 basis, double-FP32 products)."""
    from paper_2504_10096_gb300 import bse
    sizes = [150, 333, 129, 500, 257]
    nev = 6
    probs = [problem(n, dtype, seed=100 + n) for n in sizes]
    bs = bse.BatchedSolver([torch.from_numpy(a).cuda() for a, _ in probs],
                           [torch.from_numpy(b).cuda() for _, b in probs], mixed=dtype == "c64")
    vals, vecs, nconv = bs.solve(nev, tol=tol, vectors=True)
    for i, (a, b) in enumerate(probs):
        om, _, _ = O.ph_lowest(a.astype(np.complex128), b.astype(np.complex128), nev)
        assert nconv[i] == nev
        np.testing.assert_allclose(vals[i], om, rtol=rtol, atol=0)
        Z = vecs[i].cpu().numpy().astype(np.complex128)
        n = sizes[i]
        res = O.relative_residuals_ph(a, b, vals[i], Z[:n], Z[n:])
        assert res.max() < (1e-10 if dtype == "c128" else 1e-5)   # complex64 vectors as returned
        assert bs.residuals(i).max() <= tol                        # the solver's FP64 check
    bs.close()
