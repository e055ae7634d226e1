"""GB300 (sm_103a) multigrid-preconditioned CG for the HPCG 27-point operator.

Python face of the C ABI in include/hpcg.h (Scolari & Yzelman, "Effective
implementation of the High Performance Conjugate Gradient benchmark on
GraphBLAS").  This layer only marshals arguments: device memory comes from
torch tensors, streams from torch's current stream, and every step of the
solve runs in the library's CUDA kernels.  There is no CPU fallback: without
the built library, or without a GPU, the calls raise.
"""
from .binding import (HpcgProblem, HpcgBatch, HpcgEll, HpcgSplit, HpcgSolve, hpcg_solve, launch_count)  # noqa: F401
from ._lib import HpcgError, FP64, MIXED  # noqa: F401
