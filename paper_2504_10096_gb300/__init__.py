"""GB300 (sm_103a) iterative Bethe-Salpeter eigensolver.

The solver itself is the CUDA library libbse.so (C ABI in include/bse.h);
`paper_2504_10096_gb300.bse` is its thin Python binding.  Importing this
package does not load the library; the first solver call does, and fails
loudly if it has not been built.
"""
__all__ = ["bse", "build"]
