"""Pins of the oracle's Gauss-Seidel colour steps, smoother and V-cycle.

Listing 2/3 (masked mxv then elementwise update per colour), the symmetric
reading of the smoother (forward colours then backward), Listing 1 (V-cycle).
The pins restate the mathematics through dense textbook routines (triangular
solves on the colour-sorted matrix P^T A P of Section III-A).
"""
import numpy as np
import pytest

from oracle import OracleProblem
from tests import dense_ref as D


def _rand(n, seed):
    return np.random.default_rng(seed).standard_normal(n)


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 5, 7), (2, 2, 2)])
def test_colour_step_zeroes_that_colours_residual(dims):
    p = OracleProblem(*dims, levels=1)
    A = p.csr()
    col = p.colors()
    r, z = _rand(p.n(), 1), _rand(p.n(), 2)
    for k in range(8):
        zn = p.rbgs_color_step(k, r, z)
        res = r - A @ zn
        m = col == k
        assert np.abs(res[m]).max() <= 1e-13 * np.abs(r).max() * 30
        np.testing.assert_array_equal(zn[~m], z[~m])  # other colours untouched
        z = zn


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 5, 7), (6, 2, 4)])
def test_forward_sweep_is_gauss_seidel_on_colour_sorted_matrix(dims):
    p = OracleProblem(*dims, levels=1, symmetric=False)
    A = p.csr().toarray()
    r, z0 = _rand(p.n(), 3), _rand(p.n(), 4)
    z = p.rbgs(r, z0)
    zref = D.gs_forward_sorted(A, p.colors(), r, z0)
    np.testing.assert_allclose(z, zref, rtol=0, atol=1e-13 * np.abs(zref).max())


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 5, 7)])
def test_symmetric_sweep_is_forward_then_backward(dims):
    p = OracleProblem(*dims, levels=1)
    A = p.csr().toarray()
    r, z0 = _rand(p.n(), 5), _rand(p.n(), 6)
    z = p.rbgs(r, z0)
    zf = D.gs_forward_sorted(A, p.colors(), r, z0)
    zref = D.gs_backward_sorted(A, p.colors(), r, zf)
    np.testing.assert_allclose(z, zref, rtol=0, atol=1e-13 * np.abs(zref).max())


def _operator_matrix(apply, n):
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = apply(e)
    return M


def test_symmetric_smoother_is_symmetric_forward_only_is_not():
    # the HPCG rules require the replacement smoother to pass a symmetry test
    dims = (4, 4, 4)
    ps = OracleProblem(*dims, levels=1)
    pf = OracleProblem(*dims, levels=1, symmetric=False)
    n = ps.n()
    Ms = _operator_matrix(lambda e: ps.rbgs(e, np.zeros(n)), n)
    Mf = _operator_matrix(lambda e: pf.rbgs(e, np.zeros(n)), n)
    asym_s = np.abs(Ms - Ms.T).max() / np.abs(Ms).max()
    asym_f = np.abs(Mf - Mf.T).max() / np.abs(Mf).max()
    assert asym_s < 1e-13
    assert asym_f > 1e-2


@pytest.mark.parametrize("dims,levels", [((8, 8, 8), 3), ((4, 6, 8), 2), ((8, 8, 8), 1), ((8, 4, 8), 2)])
def test_vcycle_matches_dense_listing1(dims, levels):
    p = OracleProblem(*dims, levels=levels)
    As = [p.csr(l).toarray() for l in range(levels)]
    cols = [p.colors(l) for l in range(levels)]
    Rs = [D.injection_matrix(p.n(l), p.f2c(l)) for l in range(levels - 1)]
    r = _rand(p.n(), 7)
    z = p.mg(r)
    zref = D.dense_vcycle(As, cols, Rs, r)
    np.testing.assert_allclose(z, zref, rtol=0, atol=1e-12 * np.abs(zref).max())


def test_vcycle_with_kappa_matches_dense_listing1():
    kappa = np.random.default_rng(21).uniform(0, 1, 512)
    p = OracleProblem(8, 8, 8, levels=3, kappa=kappa)
    As = [p.csr(l).toarray() for l in range(3)]
    cols = [p.colors(l) for l in range(3)]
    Rs = [D.injection_matrix(p.n(l), p.f2c(l)) for l in range(2)]
    r = _rand(p.n(), 8)
    np.testing.assert_allclose(p.mg(r), D.dense_vcycle(As, cols, Rs, r), rtol=0, atol=1e-12 * 10)


def test_vcycle_preconditioner_is_spd():
    p = OracleProblem(4, 4, 8, levels=2)
    n = p.n()
    M = _operator_matrix(lambda e: p.mg(e), n)
    assert np.abs(M - M.T).max() <= 1e-13 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_vcycle_is_linear():
    p = OracleProblem(8, 8, 8, levels=3)
    a, b = _rand(p.n(), 9), _rand(p.n(), 10)
    lhs = p.mg(2.0 * a - 3.0 * b)
    rhs = 2.0 * p.mg(a) - 3.0 * p.mg(b)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12 * np.abs(rhs).max())


def _dense_smooth(A, cols, r, z, symmetric):
    z = D.gs_forward_sorted(A, cols, r, z)
    return D.gs_backward_sorted(A, cols, r, z) if symmetric else z


@pytest.mark.parametrize("kappa_seed", [None, 22])
def test_coarse_levels_receive_listing1_inputs(kappa_seed):
    """Every coarse level gets r_c = R (r - A z) after the pre-smoother and starts
    from z_c = 0, also on a second call whose buffers hold the first call's
    values.  The forward-only sweep is used: with it the restricted residual is
    of the order of the residual itself (see the next test for why the
    symmetric sweep leaves only rounding there)."""
    kappa = None if kappa_seed is None else np.random.default_rng(kappa_seed).uniform(0, 1, 512)
    p = OracleProblem(8, 8, 8, levels=3, kappa=kappa, symmetric=False)
    As = [p.csr(l).toarray() for l in range(3)]
    cols = [p.colors(l) for l in range(3)]
    Rs = [D.injection_matrix(p.n(l), p.f2c(l)) for l in range(2)]
    p.mg(_rand(p.n(), 23))  # leaves stale values on every coarse level
    r = _rand(p.n(), 24)
    p.mg(r)
    for l in range(1, 3):
        z = _dense_smooth(As[l - 1], cols[l - 1], r, np.zeros(p.n(l - 1)), False)
        rc = Rs[l - 1] @ (r - As[l - 1] @ z)
        rc_o, zc_o = p.coarse_state(l)
        assert np.abs(rc).max() > 0.1 * np.abs(r - As[l - 1] @ z).max()
        np.testing.assert_allclose(rc_o, rc, rtol=0, atol=1e-12 * np.abs(rc).max())
        zc = D.dense_vcycle(As[l:], cols[l:], Rs[l:], rc, symmetric=False)
        np.testing.assert_allclose(zc_o, zc, rtol=0, atol=1e-12 * np.abs(zc).max())
        r = rc


@pytest.mark.parametrize("symmetric", [True, False])
def test_vcycle_equals_two_fine_sweeps(symmetric):
    """A property of Listing 1 with this smoother and injection, not of the code:
    refinement writes only the all-even points, which form colour 0, and the
    post-smoother starts by recomputing colour 0 from its neighbours alone, so
    the coarse correction is overwritten (up to rounding); with the symmetric
    sweep the restricted residual is itself rounding, because the pre-smoother
    ends with colour 0."""
    p = OracleProblem(16, 16, 16, levels=4, symmetric=symmetric)
    r = _rand(p.n(), 25)
    z = p.mg(r)
    z2 = p.rbgs(r, p.rbgs(r, np.zeros(p.n())))
    assert np.abs(z - z2).max() <= 1e-14 * np.abs(z).max()
    rc, zc = p.coarse_state(1)
    res = np.abs(r - p.spmv(p.rbgs(r, np.zeros(p.n())))).max()
    if symmetric:
        assert np.abs(rc).max() <= 1e-13 * res
    else:
        assert np.abs(rc).max() > 0.1 * res and np.abs(zc).max() > 0
