"""The largest grid the block-floating-point V-cycle runs at full line length,
384^3 (56.6 M rows, 4 levels down to 48^3), against the oracle where it can
follow: SpMV rows sampled one by one (Section II-C), the pre-smoothing stage's
restricted residual at sampled injected points (Listing 1, Section II-F),
every coarse level's z against Listing 1 run by the oracle from the GPU's own
r_l, the exact scaling of the V-cycle by powers of two (block floating point
moves exponents only), and a CG solve whose recurrence residual matches the
true one."""
import numpy as np
import pytest
import torch

from hpcg_inputs import normal
from oracle import OracleProblem, spmv_rows
from tests.gpu_util import TOL64, dev, host, need_gpu, normwise

pytestmark = pytest.mark.gpu

N = 384
LEVELS = 4


@pytest.fixture(scope="module")
def grid():
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    return HpcgProblem(N, N, N, levels=LEVELS)


def test_largest_grid_spmv_sampled(grid):
    n = N ** 3
    x = normal(n, 401)
    y = host(grid.spmv(dev(x)))
    rng = np.random.default_rng(402)
    rows = np.concatenate([rng.integers(0, n, 20000), [0, N - 1, n - 1, n - N, N * N * (N // 2) + N * 7 + 5]])
    assert normwise(y[rows], spmv_rows(N, N, N, rows, x)) <= TOL64


def test_largest_grid_restriction_sampled(grid):
    """After the finest level's pre-smoothing, r_1 at coarse point c is
    (r_0 - A z_0) at the fine point c injects from, with z_0 the pre-smoothed
    finest z the stage leaves."""
    n = N ** 3
    r0 = normal(n, 403)
    grid.mg_stage(0, "pre", dev(r0), torch.zeros(n, dtype=torch.float64, device="cuda"))
    _, z0 = grid.get_level_vectors(0, r=False)
    r1, _ = grid.get_level_vectors(1, z=False)
    z0, r1 = host(z0), host(r1)
    nc = N // 2
    rng = np.random.default_rng(404)
    cs = np.concatenate([rng.integers(0, nc ** 3, 5000), [0, nc ** 3 - 1]])
    xc, yc, zc = cs % nc, (cs // nc) % nc, cs // (nc * nc)
    fine = 2 * xc + N * (2 * yc + N * 2 * zc)
    ref = r0[fine] - spmv_rows(N, N, N, fine, z0)
    # each point against the magnitudes it sums: |r_i| and sum_j |a_ij z_j|
    # (26 |z_i| plus the 26 neighbours' |z_j| = 52 |z_i| - (A |z|)_i)
    scale = np.maximum(np.abs(r0[fine]), 52 * np.abs(z0[fine]) - spmv_rows(N, N, N, fine, np.abs(z0)))
    assert np.all(np.abs(r1[cs] - ref) <= 1e-12 * scale)


def test_largest_grid_coarse_levels_and_scaling(grid):
    n = N ** 3
    r = dev(normal(n, 405))
    z = host(grid.mg_vcycle(r))
    o = OracleProblem(N >> 1, N >> 1, N >> 1, levels=LEVELS - 1)
    for l in range(1, LEVELS):
        rl, zl = grid.get_level_vectors(l)
        assert normwise(host(zl), o.mg(host(rl), l - 1)) <= TOL64, l
    # z = M r is exactly linear under scaling by powers of two
    for s in (2.0, 0.25):
        np.testing.assert_array_equal(host(grid.mg_vcycle(r * s)), z * s)


def test_largest_grid_solve_residuals(grid):
    b = grid.get_rhs()
    x, st = grid.pcg_solve(b, max_iters=20, tol=0.0)
    h = np.asarray(st.history)
    assert st.iters == 20 and h[-1] < 0.1 * h[0]
    true = float(torch.linalg.norm(b - grid.spmv(x)) / torch.linalg.norm(b))
    assert abs(true - h[-1]) <= 1e-6 * h[-1] + 1e-14
    # (x is not held against ones point by point: b = A 1 is zero off the
    # boundary, and 20 iterations have not carried the solution 80 and more
    # points in, where the oracle's values are tiny and the block-floating-
    # point V-cycle's, below 2^-56 of the neighbouring lines', are zero)
    assert bool(torch.isfinite(x).all()) and float((x - 1.0).abs().max()) <= 1.0
