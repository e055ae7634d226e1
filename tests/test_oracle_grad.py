"""Pins of the oracle's differentiable solve (gradient w.r.t. b and the
diagonal field kappa), by central finite differences (h = 1e-6) and by a
dense adjoint built with numpy.linalg.solve, on an 8^3 grid."""
import numpy as np

from oracle import OracleProblem, solve_and_grad
from hpcg_inputs import differentiable_inputs


def _loss(dims, levels, kappa, b, xt):
    p = OracleProblem(*dims, levels=levels, kappa=kappa)
    x, _ = p.pcg(b, max_iters=500, tol=1e-15)
    return 0.5 * float((x - xt) @ (x - xt))


def test_grad_vs_dense_adjoint_and_finite_differences():
    dims, levels = (8, 8, 8), 3
    n = 512
    kappa, b, xt = differentiable_inputs(n, seed=4)
    x, loss, gb, gk = solve_and_grad(dims, levels, kappa, b, xt)
    A = OracleProblem(*dims, levels=1, kappa=kappa).csr().toarray()
    xd = np.linalg.solve(A, b)
    lam = np.linalg.solve(A, xd - xt)
    np.testing.assert_allclose(x, xd, rtol=0, atol=1e-12 * np.abs(xd).max())
    np.testing.assert_allclose(gb, lam, rtol=0, atol=1e-10 * np.abs(lam).max())
    np.testing.assert_allclose(gk, -lam * xd, rtol=0, atol=1e-10 * np.abs(lam * xd).max())
    h = 1e-6
    # central differences: rounding error about eps * loss / h dominates the
    # O(h^2) truncation error at this step size
    fd_tol = 8 * np.finfo(float).eps * loss / h
    for i in [0, 7, 100, 255, 511]:
        e = np.zeros(n)
        e[i] = h
        fd_b = (_loss(dims, levels, kappa, b + e, xt) - _loss(dims, levels, kappa, b - e, xt)) / (2 * h)
        fd_k = (_loss(dims, levels, kappa + e, b, xt) - _loss(dims, levels, kappa - e, b, xt)) / (2 * h)
        assert abs(fd_b - gb[i]) <= fd_tol + 1e-6 * abs(gb[i])
        assert abs(fd_k - gk[i]) <= fd_tol + 1e-6 * abs(gk[i])
