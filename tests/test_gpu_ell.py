"""The operator materialised as a sliced-ELL matrix with rows grouped by colour
(P^T A P, Section III-A) against the oracle: the permutation and the stored
matrix exactly, the exact-arithmetic kernels bit for bit (SpMV, every colour
phase, the smoother, the V-cycle), the fused-multiply-add kernels to the FP64
tolerance, the colour-sorted and natural-order layouts bit-identical, PCG
histories, and sampled rows at 192^3."""
import numpy as np
import pytest
import torch

from hpcg_inputs import normal
from oracle import OracleProblem, spmv_rows
from tests.gpu_util import TOL64, dev, host, need_gpu, normwise

pytestmark = pytest.mark.gpu

# grids: even and odd coarse dimensions, row counts that are not multiples of 32
GRIDS = [((16, 16, 16), 4), ((6, 10, 4), 2), ((24, 8, 16), 3), ((2, 2, 2), 1), ((5, 3, 7), 1)]


def _ell(dims, levels, sorted_=True, exact=False, bf16=False):
    from paper_2304_08232_gb300 import HpcgEll
    need_gpu()
    return HpcgEll(*dims, levels=levels, colour_sorted=sorted_, exact=exact, bf16_values=bf16)


@pytest.mark.parametrize("dims,levels", GRIDS)
@pytest.mark.parametrize("sorted_", [True, False])
def test_permutation_groups_rows_by_colour(dims, levels, sorted_):
    e = _ell(dims, levels, sorted_)
    o = OracleProblem(*dims, levels=levels)
    for l in range(levels):
        col = o.colors(l)
        perm = host(e.permutation(l))
        n, slices, cstart = e.level_info(l)
        assert n == o.n(l) and slices == (n + 31) // 32
        if sorted_:
            np.testing.assert_array_equal(perm, np.argsort(col, kind="stable"))
            np.testing.assert_array_equal(np.diff(cstart), np.bincount(col, minlength=8))
            assert cstart[0] == 0 and cstart[8] == n
        else:
            np.testing.assert_array_equal(perm, np.arange(n))


@pytest.mark.parametrize("dims,levels", [((6, 4, 8), 2), ((5, 3, 7), 1), ((16, 16, 16), 1)])
@pytest.mark.parametrize("sorted_", [True, False])
def test_stored_matrix_is_the_permuted_operator(dims, levels, sorted_):
    e = _ell(dims, levels, sorted_)
    o = OracleProblem(*dims, levels=levels)
    for l in range(levels):
        n = o.n(l)
        perm = host(e.permutation(l)).astype(np.int64)
        colv, valv = (host(t) for t in e.matrix(l))
        p = np.arange(n)
        slots = ((p[:, None] // 32) * 27 + np.arange(27)[None, :]) * 32 + (p[:, None] % 32)
        C, V = colv[slots].astype(np.int64), valv[slots]
        # rebuild P^T A P and compare with the oracle's CRS matrix, permuted
        A = o.csr(l).toarray()
        B = np.zeros((n, n))
        np.add.at(B, (np.repeat(p, 27), C.ravel()), V.ravel())
        np.testing.assert_array_equal(B, A[np.ix_(perm, perm)])
        # used slots first, in ascending natural column; padding: value 0 on the own column
        nnz = o.row_nnz(l)[perm]
        used = np.arange(27)[None, :] < nnz[:, None]
        assert np.all(V[used] != 0) and np.all(V[~used] == 0)
        assert np.all(C[~used] == np.broadcast_to(p[:, None], C.shape)[~used])
        nat = np.where(used, perm[C], np.iinfo(np.int64).max)
        assert np.all(np.diff(nat, axis=1)[used[:, 1:]] > 0)


@pytest.mark.parametrize("dims,levels", GRIDS)
@pytest.mark.parametrize("sorted_", [True, False])
def test_exact_kernels_reproduce_the_oracle_bitwise(dims, levels, sorted_):
    e = _ell(dims, levels, sorted_, exact=True)
    o = OracleProblem(*dims, levels=levels)
    for l in range(levels):
        n = o.n(l)
        x, r, z0 = normal(n, 10 + l), normal(n, 20 + l), normal(n, 30 + l)
        st = lambda v: e.to_stored(dev(v), l)  # noqa: E731
        nat = lambda t: host(e.to_natural(t, l))  # noqa: E731
        np.testing.assert_array_equal(nat(e.spmv(st(x), l)), o.spmv(x, l))
        z = st(z0)
        zo = z0.copy()
        for k in range(8):
            e.rbgs_color(st(r), z, k, l)
            zo = o.rbgs_color_step(k, r, zo, l)
            np.testing.assert_array_equal(nat(z), zo)
        np.testing.assert_array_equal(nat(e.rbgs(st(r), st(z0), l)), o.rbgs(r, z0, l))
    r = normal(o.n(0), 40)
    np.testing.assert_array_equal(host(e.to_natural(e.mg_vcycle(e.to_stored(dev(r))))), o.mg(r))


@pytest.mark.parametrize("dims,levels", GRIDS[:3])
def test_fma_kernels_within_fp64_tolerance_and_layout_independent(dims, levels):
    es, en = _ell(dims, levels, True), _ell(dims, levels, False)
    o = OracleProblem(*dims, levels=levels)
    n = o.n(0)
    x, r = normal(n, 50), normal(n, 51)
    ys = host(es.to_natural(es.spmv(es.to_stored(dev(x)))))
    yn = host(en.spmv(dev(x)))
    assert normwise(ys, o.spmv(x)) <= TOL64
    np.testing.assert_array_equal(ys, yn)  # same per-row arithmetic in both layouts
    zs = host(es.to_natural(es.mg_vcycle(es.to_stored(dev(r)))))
    zn = host(en.mg_vcycle(dev(r)))
    assert normwise(zs, o.mg(r)) <= TOL64
    np.testing.assert_array_equal(zs, zn)


@pytest.mark.parametrize("dims,levels", [((16, 16, 16), 4), ((6, 10, 4), 2), ((5, 3, 7), 1)])
@pytest.mark.parametrize("exact", [True, False])
def test_bf16_values_give_the_same_bits(dims, levels, exact):
    """26, -1 and 0 are exact in BF16: the BF16-valued matrix stores the same
    operator in a quarter of the value bytes and every level call and the solve
    give the same bits as with FP64 values."""
    e8, e2 = _ell(dims, levels, True, exact), _ell(dims, levels, True, exact, bf16=True)
    assert e2.nbytes() < e8.nbytes()
    for l in range(levels):
        c8, v8 = (host(t) for t in e8.matrix(l))
        c2, v2 = (host(t) for t in e2.matrix(l))
        np.testing.assert_array_equal(c2, c8)
        np.testing.assert_array_equal(v2, v8)
        n = e8.level_info(l)[0]
        x = dev(normal(n, 56 + l))
        np.testing.assert_array_equal(host(e2.spmv(x, l)), host(e8.spmv(x, l)))
        r, z = dev(normal(n, 60 + l)), dev(normal(n, 64 + l))
        np.testing.assert_array_equal(host(e2.rbgs(r, z.clone(), l)), host(e8.rbgs(r, z.clone(), l)))
    n = e8.n
    r = dev(normal(n, 68))
    np.testing.assert_array_equal(host(e2.mg_vcycle(r)), host(e8.mg_vcycle(r)))
    b = dev(normal(n, 69))
    x8, s8 = e8.pcg_solve(b, max_iters=20, tol=0.0)
    x2, s2 = e2.pcg_solve(b, max_iters=20, tol=0.0)
    np.testing.assert_array_equal(host(x2), host(x8))
    np.testing.assert_array_equal(np.asarray(s2.history), np.asarray(s8.history))


@pytest.mark.parametrize("exact", [True, False])
def test_pcg_history_matches_oracle(exact):
    dims, levels = (16, 16, 16), 4
    e = _ell(dims, levels, True, exact=exact)
    o = OracleProblem(*dims, levels=levels)
    b = o.rhs()
    x, st = e.pcg_solve(dev(b), max_iters=50, tol=0.0)
    xo, ho = o.pcg(b, max_iters=50, tol=0.0)
    h = np.asarray(st.history)
    assert st.iters == 50 and len(h) == 50
    live = ho > 1e-11
    assert np.max(np.abs(h[live] - ho[live]) / ho[live]) <= 1e-6
    assert normwise(host(x), xo) <= 1e-10
    assert np.abs(host(x) - 1.0).max() <= 1e-9  # b = A * ones


def test_pcg_to_tolerance_matches_matrix_free_iterations():
    from paper_2304_08232_gb300 import HpcgProblem
    dims, levels = (32, 24, 40), 4
    n = int(np.prod(dims))
    e = _ell(dims, levels, True)
    g = HpcgProblem(*dims, levels=levels)
    b = normal(n, 52)
    x, st = e.pcg_solve(dev(b), max_iters=200, tol=1e-9)
    xg, sg = g.pcg_solve(dev(b), max_iters=200, tol=1e-9)
    assert st.converged and sg.converged and abs(st.iters - sg.iters) <= 1
    assert normwise(host(x), host(xg)) <= 1e-8
    # x0 goes through the permutation and back unchanged when no iteration runs
    x2, st2 = e.pcg_solve(dev(b), x0=x, max_iters=0, tol=0.0)
    assert st2.iters == 0
    np.testing.assert_array_equal(host(x2), host(x))


def test_fullsize_192cubed_sampled_rows():
    """192^3: sampled rows of the SpMV against the oracle's row evaluation,
    the layouts bit-identical, and the 50-iteration solve of b = A * ones
    against the matrix-free solve."""
    dims = (192, 192, 192)
    n = int(np.prod(dims))
    es = _ell(dims, 4, True)
    x = normal(n, 53)
    y = host(es.to_natural(es.spmv(es.to_stored(dev(x)))))
    rows = np.random.default_rng(54).choice(n, 4096, replace=False)
    np.testing.assert_allclose(y[rows], spmv_rows(*dims, rows, x), rtol=0, atol=1e-12 * np.abs(y).max())
    en = _ell(dims, 4, False)
    np.testing.assert_array_equal(host(en.spmv(dev(x))), y)
    del en
    # 50 iterations of b = A * ones leave an error of about 3e-2; the same as
    # the matrix-free solve (same method, other rounding) to 1e-10
    from paper_2304_08232_gb300 import HpcgProblem
    b = torch.as_tensor(spmv_rows(*dims, np.arange(n, dtype=np.int64), np.ones(n)), device="cuda")
    xs, st = es.pcg_solve(b, max_iters=50, tol=0.0)
    xg, sg = HpcgProblem(*dims, levels=4).pcg_solve(b, max_iters=50, tol=0.0)
    assert st.iters == 50
    assert normwise(host(xs), host(xg)) <= 1e-10
    h, hg = np.asarray(st.history), np.asarray(sg.history)
    assert np.max(np.abs(h - hg) / hg) <= 1e-8


def test_argument_errors():
    from paper_2304_08232_gb300 import HpcgEll, HpcgError
    need_gpu()
    with pytest.raises(HpcgError):
        HpcgEll(6, 6, 6, levels=3)  # 6 not divisible by 4
    e = HpcgEll(8, 8, 8, levels=2)
    r = dev(normal(512, 55))
    with pytest.raises(HpcgError):
        e.rbgs_color(r, r.clone(), 8)
    with pytest.raises(HpcgError):
        e.spmv(r, level=2)
    with pytest.raises(HpcgError):
        e.spmv(r, out=r)
