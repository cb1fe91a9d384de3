"""Seeded synthetic inputs shared by the oracle and the CUDA path (no solver arithmetic)."""
from .bse_matrices import *  # noqa: F401,F403
