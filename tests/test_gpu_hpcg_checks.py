"""HPCG's symmetry test on the GPU path (Section III-A: the smoother replacing
symmetric Gauss-Seidel must keep the preconditioner symmetric): x'Ay = y'Ax
and x'My = y'Mx for random x, y, to rounding, with the symmetric smoother in
both storage forms of the V-cycle; the forward-only ablation is not
symmetric."""
import numpy as np
import pytest
import torch

from hpcg_inputs import normal
from tests.gpu_util import dev, need_gpu

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


@pytest.mark.parametrize("block_fp", [True, False])
@pytest.mark.parametrize("dims,levels", [((32, 32, 32), 4), ((48, 32, 64), 4), ((16, 24, 8), 2)])
def test_operator_and_preconditioner_are_symmetric(dims, levels, block_fp):
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    n = int(np.prod(dims))
    g = HpcgProblem(*dims, levels=levels, block_fp=block_fp)
    x, y = dev(normal(n, 43)), dev(normal(n, 44))
    scale = float(torch.linalg.norm(x) * torch.linalg.norm(y))
    dA = abs(float(torch.dot(x, g.spmv(y)) - torch.dot(y, g.spmv(x))))
    assert dA <= 64 * EPS * scale * 52
    dM = abs(float(torch.dot(x, g.mg_vcycle(y)) - torch.dot(y, g.mg_vcycle(x))))
    assert dM <= 64 * EPS * scale


def test_forward_only_preconditioner_is_not_symmetric():
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    dims = (32, 32, 32)
    n = int(np.prod(dims))
    g = HpcgProblem(*dims, levels=4, symmetric=False)
    x, y = dev(normal(n, 45)), dev(normal(n, 46))
    scale = float(torch.linalg.norm(x) * torch.linalg.norm(y))
    dM = abs(float(torch.dot(x, g.mg_vcycle(y)) - torch.dot(y, g.mg_vcycle(x))))
    assert dM >= 1e-6 * scale
