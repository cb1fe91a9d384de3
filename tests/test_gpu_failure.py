"""Failure detection on the GPU without a GPU fault: a bounded device wait on
an mbarrier that nothing completes gives up with an error status, and the
CUDA context stays usable for the next call."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import problem, rand_block, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_bounded_wait_expires_and_context_survives():
    from paper_2504_10096_gb300 import bse
    rc, expired = bse.bse_selftest_bounded_wait(0)
    assert rc == bse.BSE_OK and expired == 1
    rc, expired = bse.bse_selftest_bounded_wait(1)
    assert rc == bse.BSE_OK and expired == 0
    # the context still works: a structured product against the oracle
    A, B = problem(150, "c128", seed=91)
    s = bse.Solver(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    X = rand_block(150, 1, "c128", seed=9)
    Y = s.apply(bse.BSE_OP_MPLUS, torch.from_numpy(X).cuda()).cpu().numpy()
    assert rel(Y, O.apply_mplus(A, B, X)) < 1e-13
    s.close()
