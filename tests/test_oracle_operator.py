"""Pins of the oracle's operator, colouring and transfer maps (CPU only).

Operator: Section II-B/II-C (27-point stencil, 8..27 nonzeros per row);
A_diag: Section III-A; greedy colouring with eight colours: Section III-A;
straight injection and its transpose: Sections II-F and III-B.
"""
import numpy as np
import pytest

from oracle import OracleProblem
from oracle.oracle import row_entries
from oracle import spmv_rows
from tests import dense_ref as D

GRIDS = [(2, 2, 2), (3, 5, 7), (4, 4, 4), (5, 3, 2), (6, 4, 8)]


@pytest.mark.parametrize("dims", GRIDS + [(16, 16, 16)])
def test_nnz_closed_form(dims):
    nx, ny, nz = dims
    p = OracleProblem(nx, ny, nz, levels=1)
    assert p.nnz() == (3 * nx - 2) * (3 * ny - 2) * (3 * nz - 2)
    rn = p.row_nnz()
    # rows with k interior coordinates have 2^(3-k) * 3^k entries
    inner = [max(d - 2, 0) for d in dims]
    expect = {
        8: 8,
        12: 4 * sum(inner),
        18: 2 * (inner[0] * inner[1] + inner[1] * inner[2] + inner[0] * inner[2]),
        27: inner[0] * inner[1] * inner[2],
    }
    for k, v in expect.items():
        assert int((rn == k).sum()) == v
    assert set(np.unique(rn)) <= {8, 12, 18, 27}


@pytest.mark.parametrize("dims", GRIDS)
def test_operator_is_kronecker_form(dims):
    p = OracleProblem(*dims, levels=1)
    A = p.csr().toarray()
    np.testing.assert_array_equal(A, D.kron_operator(*dims))


def test_operator_with_kappa_is_kronecker_form():
    dims = (3, 4, 5)
    kappa = np.linspace(0.0, 1.0, 60)
    p = OracleProblem(*dims, levels=1, kappa=kappa)
    A = p.csr().toarray()
    np.testing.assert_array_equal(A, D.kron_operator(*dims, kappa=kappa))
    np.testing.assert_array_equal(p.diag(), 26.0 + kappa)


@pytest.mark.parametrize("dims", [(3, 4, 5), (4, 4, 4), (2, 6, 3)])
def test_spectrum_closed_form(dims):
    A = OracleProblem(*dims, levels=1).csr().toarray()
    ev = np.linalg.eigvalsh(A)
    np.testing.assert_allclose(ev, D.kron_eigenvalues(*dims), rtol=0, atol=1e-10)
    assert ev.min() > 0  # SPD


def test_columns_ascending_and_diag_vector():
    p = OracleProblem(5, 4, 3, levels=1)
    A = p.csr()
    for i in range(A.shape[0]):
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
    np.testing.assert_array_equal(p.diag(), A.diagonal())
    np.testing.assert_array_equal(p.diag(), np.full(60, 26.0))


def test_symmetry():
    p = OracleProblem(6, 5, 4, levels=1)
    rng = np.random.default_rng(11)
    x, y = rng.standard_normal(p.n()), rng.standard_normal(p.n())
    lhs = y @ p.spmv(x)
    rhs = x @ p.spmv(y)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_rhs_gives_unit_solution_rowsums():
    # b = A * ones has b_i = 26 - (nnz_i - 1) = 27 - nnz_i.
    p = OracleProblem(5, 6, 7, levels=1)
    np.testing.assert_array_equal(p.rhs(), 27.0 - p.row_nnz())


def test_spmv_matches_library_product():
    p = OracleProblem(7, 6, 5, levels=1)
    x = np.random.default_rng(3).standard_normal(p.n())
    np.testing.assert_allclose(p.spmv(x), p.csr() @ x, rtol=0, atol=1e-12)
    rows = np.array([0, 1, 41, 100, p.n() - 1])
    np.testing.assert_allclose(spmv_rows(7, 6, 5, rows, x), (p.csr() @ x)[rows], rtol=0, atol=1e-12)


def test_row_generator_corner_and_interior():
    cols, vals = row_entries(4, 4, 4, 0)
    assert list(cols) == [0, 1, 4, 5, 16, 17, 20, 21]
    assert list(vals) == [26.0] + [-1.0] * 7
    i = 1 + 4 * (1 + 4 * 1)
    cols, vals = row_entries(4, 4, 4, i)
    assert len(cols) == 27 and vals[13] == 26.0 and cols[13] == i


@pytest.mark.parametrize("dims", GRIDS + [(16, 16, 16), (3, 3, 3)])
def test_greedy_colouring_is_parity_and_valid(dims):
    p = OracleProblem(*dims, levels=1)
    col = p.colors()
    A = p.csr().tocoo()
    off = A.row != A.col
    assert np.all(col[A.row[off]] != col[A.col[off]])          # valid
    np.testing.assert_array_equal(col, D.parity_colors(*dims))  # closed form
    assert p.ncolors() == 8


def test_eight_colours_are_necessary():
    # every 2x2x2 block is a clique of the dependence graph, so no valid
    # colouring uses fewer than eight colours: greedy is optimal here.
    A = OracleProblem(2, 2, 2, levels=1).csr().toarray()
    assert np.all(A != 0)


@pytest.mark.parametrize("dims,levels", [((8, 8, 8), 3), ((4, 6, 8), 2), ((16, 16, 16), 4), ((8, 8, 12), 3)])
def test_injection_lowest_corner(dims, levels):
    p = OracleProblem(*dims, levels=levels)
    for l in range(levels - 1):
        nxf, nyf, _ = p.dims(l)
        nxc, nyc, nzc = p.dims(l + 1)
        assert (nxc, nyc, nzc) == (p.dims(l)[0] // 2, p.dims(l)[1] // 2, p.dims(l)[2] // 2)
        f2c = p.f2c(l)
        c = np.arange(len(f2c))
        xc, yc, zc = c % nxc, (c // nxc) % nyc, c // (nxc * nyc)
        fx, fy, fz = f2c % nxf, (f2c // nxf) % nyf, f2c // (nxf * nyf)
        np.testing.assert_array_equal(fx, 2 * xc)
        np.testing.assert_array_equal(fy, 2 * yc)
        np.testing.assert_array_equal(fz, 2 * zc)
        # every injected point has colour 0 (all coordinates even)
        assert np.all(p.colors(l)[f2c] == 0)


def test_restrict_prolong_are_R_and_RT():
    p = OracleProblem(8, 8, 8, levels=3)
    rng = np.random.default_rng(5)
    for l in range(2):
        R = D.injection_matrix(p.n(l), p.f2c(l))
        np.testing.assert_array_equal(R @ R.T, np.eye(p.n(l + 1)))  # R P = I
        v = rng.standard_normal(p.n(l))
        np.testing.assert_array_equal(p.restrict(v, l), R @ v)
        zc = rng.standard_normal(p.n(l + 1))
        z = rng.standard_normal(p.n(l))
        np.testing.assert_allclose(p.prolong_add(zc, z, l), z + R.T @ zc, rtol=0, atol=0)


def test_coarse_operator_regenerated_with_injected_kappa():
    kappa = np.random.default_rng(9).uniform(0, 1, 8 * 8 * 8)
    p = OracleProblem(8, 8, 8, levels=3, kappa=kappa)
    f2c0 = p.f2c(0)
    np.testing.assert_array_equal(p.csr(1).toarray(), D.kron_operator(4, 4, 4, kappa=kappa[f2c0]))
    f2c1 = p.f2c(1)
    np.testing.assert_array_equal(p.diag(2), 26.0 + kappa[f2c0][f2c1])


@pytest.mark.parametrize("dims,levels", [((3, 4, 4), 2), ((4, 4, 4), 3), ((8, 8, 12), 4), ((1, 4, 4), 1), ((4, 4, 4), 0)])
def test_invalid_sizes_rejected(dims, levels):
    with pytest.raises(ValueError):
        OracleProblem(*dims, levels=levels)
