"""GB300-native FT-GCR(k): fault-tolerant preconditioned GCR elliptic solver
(Gillard & Benacchio, arXiv 2103.07210, Algorithm 1) as a C-ABI CUDA library
for sm_103a with a thin Python binding."""
from .ftgcr import (FP64, MIXED, NOT_CONVERGED, OK, FTGCRError, Solver, build, footprint, lib,  # noqa: F401
                    solve_batch)
