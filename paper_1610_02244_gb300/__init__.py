"""GB300 (sm_103a) two-site update for MPS algorithms (arXiv:1610.02244).

The CUDA library libtntgb.so implements the effective-Hamiltonian matvec, Lanczos,
truncated SVD, environment growth, theta formation and TEBD gates behind the C-ABI of
include/tnt_gb300.h.  ``paper_1610_02244_gb300.tnt`` is the Python API over it; importing
the package itself loads nothing, so the seeded input generators in ``synth`` stay usable
without a GPU.
"""

__all__ = ["synth", "tnt", "build"]
