"""Pins of the oracle's preconditioned CG (Section II-C; HPCG iteration order).

The iterate after k steps must be the A-norm minimiser of the error over the
preconditioned Krylov space x0 + span{M r0, (M A) M r0, ...}; the converged
solution must equal a dense direct solve; for the HPCG right-hand side the
exact solution is the vector of ones.
"""
import numpy as np
import pytest

from oracle import OracleProblem


def _krylov_minimiser(A, M, b, x0, k):
    """argmin over x0 + K_k(MA, M r0) of ||x - x*||_A, by a dense projection."""
    r0 = b - A @ x0
    V = [M @ r0]
    for _ in range(k - 1):
        V.append(M @ (A @ V[-1]))
    V = np.array(V).T
    Q, _ = np.linalg.qr(V)
    # minimise ||x0 + Q y - x*||_A  =>  (Q^T A Q) y = Q^T r0
    y = np.linalg.solve(Q.T @ A @ Q, Q.T @ r0)
    return x0 + Q @ y


def _dense_M(p):
    n = p.n()
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = p.mg(e)
    return 0.5 * (M + M.T)


@pytest.mark.parametrize("dims,levels", [((4, 4, 4), 2), ((4, 6, 8), 2)])
def test_pcg_iterates_are_krylov_minimisers(dims, levels):
    p = OracleProblem(*dims, levels=levels)
    A = p.csr().toarray()
    M = _dense_M(p)
    b = np.random.default_rng(1).standard_normal(p.n())
    x0 = np.random.default_rng(2).standard_normal(p.n())
    xs = np.linalg.solve(A, b)
    for k in range(1, 5):
        xk, _ = p.pcg(b, x0=x0, max_iters=k, tol=0.0)
        xm = _krylov_minimiser(A, M, b, x0, k)
        err = np.sqrt((xk - xm) @ A @ (xk - xm))
        scale = np.sqrt((x0 - xs) @ A @ (x0 - xs))
        assert err <= 1e-9 * scale, (k, err, scale)


def test_plain_cg_iterates_are_krylov_minimisers():
    p = OracleProblem(4, 4, 4, levels=1)
    A = p.csr().toarray()
    b = np.random.default_rng(4).standard_normal(p.n())
    x0 = np.zeros(p.n())
    for k in range(1, 6):
        xk, _ = p.pcg(b, x0=x0, max_iters=k, tol=0.0, precond=False)
        xm = _krylov_minimiser(A, np.eye(p.n()), b, x0, k)
        assert np.abs(xk - xm).max() <= 1e-10 * np.abs(xm).max()


@pytest.mark.parametrize("dims,levels", [((8, 8, 8), 3), ((4, 6, 8), 2), ((6, 6, 6), 2)])
def test_pcg_converges_to_dense_solution(dims, levels):
    p = OracleProblem(*dims, levels=levels)
    A = p.csr().toarray()
    b = np.random.default_rng(6).standard_normal(p.n())
    x, hist = p.pcg(b, max_iters=100, tol=1e-14)
    xs = np.linalg.solve(A, b)
    assert np.abs(x - xs).max() <= 1e-12 * np.abs(xs).max()
    assert hist[-1] <= 1e-14


def test_pcg_history_is_true_relative_residual_and_anorm_monotone():
    p = OracleProblem(8, 8, 8, levels=3)
    A = p.csr()
    b = np.random.default_rng(7).standard_normal(p.n())
    xs = np.linalg.solve(A.toarray(), b)
    prev = np.inf
    _, hist = p.pcg(b, max_iters=8, tol=0.0)
    for k in range(1, 9):
        xk, _ = p.pcg(b, max_iters=k, tol=0.0)
        true_rel = np.linalg.norm(b - A @ xk) / np.linalg.norm(b)
        assert abs(true_rel - hist[k - 1]) <= 1e-10 * true_rel + 1e-15
        e = xk - xs
        anorm = np.sqrt(e @ (A @ e))
        assert anorm <= prev * (1 + 1e-12)
        prev = anorm


def test_hpcg_rhs_exact_solution_is_ones():
    p = OracleProblem(16, 16, 16, levels=4)
    x, hist = p.pcg(p.rhs(), max_iters=50, tol=0.0)
    assert len(hist) == 50
    assert np.abs(x - 1.0).max() <= 1e-12
    assert hist[19] < 1e-12


def test_tolerance_stop():
    p = OracleProblem(8, 8, 8, levels=3)
    _, hist = p.pcg(p.rhs(), max_iters=100, tol=1e-6)
    assert hist[-1] <= 1e-6 and (len(hist) == 1 or hist[-2] > 1e-6)
