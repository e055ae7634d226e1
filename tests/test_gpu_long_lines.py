"""Long x-lines against the oracle: 256 and 320 points (the block-floating-
point V-cycle with four and five 64-point chunks per line, the SpMV line
kernels with 8 and 10 32-point chunks), 448 points (past the 384 the
block-floating-point V-cycle takes: FP64 level vectors, and an SpMV of 14
chunks, which no line kernel is built for: the one-thread-per-row kernel) and
1088 points (the same fallbacks with two levels).  Section II-C (SpMV, CG) and
Listing 1 (the V-cycle) on grids whose lines cross every register-window
boundary of the line kernels."""
import numpy as np
import pytest

from hpcg_inputs import normal, uniform
from oracle import OracleProblem
from tests.gpu_util import TOL32, TOL64, dev, host, need_gpu, normwise

pytestmark = pytest.mark.gpu

CASES = [((256, 8, 8), 3), ((320, 8, 12), 3), ((448, 8, 8), 3), ((1088, 4, 4), 2)]


def _pair(dims, levels, kappa=None, precision="fp64"):
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    g = HpcgProblem(*dims, levels=levels, precision=precision, kappa=None if kappa is None else dev(kappa))
    o = OracleProblem(*dims, levels=levels, kappa=kappa)
    return g, o


@pytest.mark.parametrize("dims,levels", CASES)
@pytest.mark.parametrize("with_kappa", [False, True])
def test_long_lines_spmv_every_level(dims, levels, with_kappa):
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 41) if with_kappa else None
    g, o = _pair(dims, levels, kappa)
    for l in range(levels):
        x = normal(o.n(l), 300 + l)
        assert normwise(host(g.spmv(dev(x), level=l)), o.spmv(x, l)) <= TOL64, l


@pytest.mark.parametrize("dims,levels", CASES)
@pytest.mark.parametrize("with_kappa", [False, True])
def test_long_lines_vcycle_and_coarse_levels(dims, levels, with_kappa):
    """The V-cycle's output, and each coarse z_l it leaves against Listing 1
    run from level l on the r_l it leaves (the final z alone does not show the
    coarse levels: the post-smoother recomputes the points they correct)."""
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 42) if with_kappa else None
    g, o = _pair(dims, levels, kappa)
    r = normal(n, 310)
    assert normwise(host(g.mg_vcycle(dev(r))), o.mg(r)) <= TOL64
    for l in range(1, levels):
        rl, zl = g.get_level_vectors(l)
        rl, zl = host(rl), host(zl)
        assert np.abs(rl).max() > 0, l
        assert normwise(zl, o.mg(rl, l)) <= TOL64, l


@pytest.mark.parametrize("dims,levels", CASES)
def test_long_lines_mixed_vcycle(dims, levels):
    g, o = _pair(dims, levels, precision="mixed")
    r = normal(int(np.prod(dims)), 320)
    assert normwise(host(g.mg_vcycle(dev(r))), o.mg(r)) <= TOL32


@pytest.mark.parametrize("dims,levels", CASES)
def test_long_lines_pcg_history(dims, levels):
    g, o = _pair(dims, levels)
    b = normal(int(np.prod(dims)), 330)
    x, st = g.pcg_solve(dev(b), max_iters=30, tol=0.0)
    xr, hr = o.pcg(b, max_iters=30, tol=0.0)
    assert st.iters == 30
    h, hr = np.asarray(st.history), np.asarray(hr)
    live = hr > 1e-11
    assert (np.abs(h[live] - hr[live]) / hr[live]).max() <= 1e-6
    assert normwise(host(x), xr) <= 1e-9


@pytest.mark.parametrize("dims", [[(320, 8, 8), (192, 8, 8), (40, 16, 8), (64, 8, 16), (8, 8, 8)],
                                  [(448, 8, 8), (96, 8, 12), (24, 8, 8)]])
def test_batch_of_mixed_line_lengths(dims):
    """A batch whose instances' lines span the register windows (each block
    takes its own instance's window) or pass the block-floating-point limit
    (448: the whole batch keeps FP64 level vectors)."""
    from paper_2304_08232_gb300 import HpcgBatch
    need_gpu()
    levels = 3
    bat = HpcgBatch(dims, levels=levels)
    offs = bat.offsets
    b = normal(bat.n, 340)
    x, sts = bat.pcg_solve(dev(b), max_iters=25, tol=0.0)
    xh = host(x)
    for i, d in enumerate(dims):
        o = OracleProblem(*d, levels=levels)
        xr, hr = o.pcg(b[offs[i]:offs[i + 1]], max_iters=25, tol=0.0)
        h, hr = np.asarray(sts[i].history), np.asarray(hr)
        assert sts[i].iters == 25
        live = hr > 1e-11
        assert (np.abs(h[live] - hr[live]) / hr[live]).max() <= 1e-6, i
        assert normwise(xh[offs[i]:offs[i + 1]], xr) <= 1e-9, i
