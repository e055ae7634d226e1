"""Full-size checks of the mixed-precision and differentiable workloads through
properties the oracle can verify at any size: the true residual recomputed by
the oracle's SpMV row by row, the error bound cond(A) * residual from the
closed-form spectrum, the adjoint equation A lambda = x - x_target, the
pointwise gradient -lambda * x, and a directional finite difference of the
loss."""
import numpy as np
import pytest
import torch

from hpcg_inputs import differentiable_inputs, mixed_precision_xtrue
from oracle import spmv_rows
from tests.dense_ref import kron_eigenvalues
from tests.gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu


def _apply(dims, x, kappa=None):
    n = int(np.prod(dims))
    return spmv_rows(*dims, np.arange(n, dtype=np.int64), x, kappa=kappa)


def test_mixed_precision_192cubed_to_1e9():
    """The mixed-precision workload: 192^3, 4 levels, b = A x_true with
    x_true ~ U[-1, 1], solved to a relative residual of 1e-9."""
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    dims = (192, 192, 192)
    n = int(np.prod(dims))
    xt = mixed_precision_xtrue(n, seed=1)
    b = _apply(dims, xt)
    g = HpcgProblem(*dims, levels=4, precision="mixed")
    x, st = g.pcg_solve(dev(b), max_iters=400, tol=1e-9)
    assert st.converged and st.rel_res <= 1e-9
    xh = host(x)
    res = np.linalg.norm(b - _apply(dims, xh)) / np.linalg.norm(b)
    assert res <= 2e-9
    ev = kron_eigenvalues(*dims)
    cond = ev[-1] / ev[0]
    assert np.linalg.norm(xh - xt) / np.linalg.norm(xt) <= cond * res * 1.01
    # the FP64 solve reaches the same tolerance in a comparable number of iterations
    g64 = HpcgProblem(*dims, levels=4)
    _, st64 = g64.pcg_solve(dev(b), max_iters=400, tol=1e-9)
    assert st64.converged and abs(st.iters - st64.iters) <= max(5, st64.iters // 10)


def test_differentiable_solve_96cubed():
    """The differentiable workload: 96^3, 4 levels, kappa ~ U[0, 1],
    b, x_target ~ N(0, 1), loss 0.5 ||x - x_target||^2."""
    from paper_2304_08232_gb300 import HpcgProblem, hpcg_solve
    need_gpu()
    dims = (96, 96, 96)
    n = int(np.prod(dims))
    kappa, b, xtarget = differentiable_inputs(n, seed=4)
    g = HpcgProblem(*dims, levels=4)
    bt = dev(b).requires_grad_(True)
    kt = dev(kappa).requires_grad_(True)
    x = hpcg_solve(bt, kt, g, max_iters=400, tol=1e-13)
    loss = 0.5 * ((x - dev(xtarget)) ** 2).sum()
    loss.backward()
    xh, lam, gk = host(x), host(bt.grad), host(kt.grad)
    # forward and adjoint equations, residuals recomputed by the oracle
    assert np.linalg.norm(b - _apply(dims, xh, kappa)) / np.linalg.norm(b) <= 1e-12
    gx = xh - xtarget
    assert np.linalg.norm(gx - _apply(dims, lam, kappa)) / np.linalg.norm(gx) <= 1e-12
    # dA/dkappa_i = e_i e_i^T, so the gradient is -lambda_i x_i at every point
    np.testing.assert_allclose(gk, -lam * xh, rtol=1e-15, atol=0)
    # directional derivative along d against a fourth-order central difference
    d = np.random.default_rng(5).standard_normal(n)
    G = float(gk @ d)
    L0 = float(loss.detach())

    def L(e):
        g.set_kappa(dev(kappa + e * d))
        xe, st = g.pcg_solve(dev(b), max_iters=400, tol=1e-13)
        assert st.converged
        return 0.5 * float(((xe - dev(xtarget)) ** 2).sum())

    eps = 1e-2
    fd = (8 * (L(eps) - L(-eps)) - (L(2 * eps) - L(-2 * eps))) / (12 * eps)
    assert abs(fd - G) <= 1e-7 * abs(G) + 64 * np.finfo(float).eps * L0 / eps
