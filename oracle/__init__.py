"""FP64 CPU oracle for the BSE eigenproblem and the Haydock spectrum --
test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
leg may import this package.  The CUDA product path never touches it.
"""
from .dense import *  # noqa: F401,F403
from .haydock import *  # noqa: F401,F403
