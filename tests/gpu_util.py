"""Helpers of the GPU parity tests."""
import numpy as np
import pytest
import torch


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def normwise(a, ref):
    """||a - ref||_inf / ||ref||_inf (0 when both vanish)."""
    den = np.abs(ref).max()
    num = np.abs(a - ref).max()
    return num / den if den > 0 else num


# FP64 kernel outputs: each output is a sum of at most 27 terms of the inputs
# (times fixed coefficients), formed in a different order than the oracle's;
# 1e-12 normwise bounds the reordering error by a wide margin for the inputs
# used here (random N(0,1) vectors, row sums of at most 27 |terms|).
TOL64 = 1e-12
# FP32 preconditioner (mixed precision): unit roundoff 6e-8, a V-cycle chains
# about 30 colour steps per level over 4 levels; 2e-5 normwise.
TOL32 = 2e-5
