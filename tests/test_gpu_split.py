"""One grid as two z-slabs with their own rows and halo planes and
colour-aware halo exchange, on one GPU, against the oracle: the slab and halo
bookkeeping, the exact-arithmetic SpMV, smoother and V-cycle bit for bit on
every level (so every halo value a colour phase reads was exchanged in time),
the exchange volume, PCG histories, and the whole-grid engine at 192^3."""
import numpy as np
import pytest
import torch

from hpcg_inputs import normal
from oracle import OracleProblem
from tests.gpu_util import TOL64, dev, host, need_gpu, normwise

pytestmark = pytest.mark.gpu

# nz divisible by 2^levels: each slab keeps a plane on the coarsest level
GRIDS = [((16, 16, 16), 4), ((6, 10, 8), 2), ((24, 8, 16), 3), ((4, 6, 2), 1), ((5, 3, 8), 1)]


def _split(dims, levels, exact=False):
    from paper_2304_08232_gb300 import HpcgSplit
    need_gpu()
    return HpcgSplit(*dims, levels=levels, exact=exact)


@pytest.mark.parametrize("dims,levels", GRIDS)
def test_slabs_and_halos(dims, levels):
    s = _split(dims, levels)
    o = OracleProblem(*dims, levels=levels)
    for l in range(levels):
        nx, ny, nz = o.dims(l)
        col = o.colors(l).reshape(nz, ny, nx)
        i0, i1 = s.info(l, 0), s.info(l, 1)
        assert i0["z"] == (0, nz // 2) and i1["z"] == (nz // 2, nz)
        for i, zh in ((i0, nz // 2), (i1, nz // 2 - 1)):
            z0, z1 = i["z"]
            assert i["own"] == nx * ny * (z1 - z0) and i["halo"] == nx * ny
            np.testing.assert_array_equal(np.diff(i["cstart"]), np.bincount(col[z0:z1].ravel(), minlength=8))
            # the halo is the neighbour's boundary plane: four colours of one z parity
            np.testing.assert_array_equal(np.diff(i["hstart"]), np.bincount(col[zh].ravel(), minlength=8))


@pytest.mark.parametrize("dims,levels", GRIDS)
def test_exact_level_calls_reproduce_the_oracle_bitwise(dims, levels):
    s = _split(dims, levels, exact=True)
    o = OracleProblem(*dims, levels=levels)
    for l in range(levels):
        n = o.n(l)
        x, r, z0 = normal(n, 60 + l), normal(n, 70 + l), normal(n, 80 + l)
        np.testing.assert_array_equal(host(s.spmv(dev(x), l)), o.spmv(x, l))
        np.testing.assert_array_equal(host(s.rbgs(dev(r), dev(z0), l)), o.rbgs(r, z0, l))
    r = normal(o.n(0), 90)
    np.testing.assert_array_equal(host(s.mg_vcycle(dev(r))), o.mg(r))


def test_colour_aware_exchange_volume():
    """A smoother application moves each halo value twice (once per sweep
    direction) plus the entering z once; a V-cycle adds colour 0 after each
    refinement.  Exchanging the whole halo after every colour would move 16x."""
    dims, levels = (16, 12, 16), 3
    s = _split(dims, levels)
    halo = lambda l: s.info(l, 0)["halo"] + s.info(l, 1)["halo"]  # noqa: E731
    n = int(np.prod(dims))
    v0, k0 = s.exchange_count()
    s.rbgs(dev(normal(n, 91)), dev(normal(n, 92)), 0)
    v1, k1 = s.exchange_count()
    assert v1 - v0 == 3 * halo(0) and k1 - k0 == 17
    s.mg_vcycle(dev(normal(n, 93)))
    v2, k2 = s.exchange_count()
    col0 = lambda l: sum(s.info(l, d)["hstart"][1] - s.info(l, d)["hstart"][0] for d in (0, 1))  # noqa: E731
    expect = sum(4 * halo(l) for l in range(levels - 1)) + 2 * halo(levels - 1) + sum(col0(l) for l in range(levels - 1))
    assert v2 - v1 == expect
    assert k2 - k1 == 32 * (levels - 1) + 16 + (levels - 1)


@pytest.mark.parametrize("exact", [True, False])
def test_pcg_history_matches_oracle(exact):
    dims, levels = (16, 16, 16), 4
    s = _split(dims, levels, exact=exact)
    o = OracleProblem(*dims, levels=levels)
    b = o.rhs()
    x, st = s.pcg_solve(dev(b), max_iters=50, tol=0.0)
    xo, ho = o.pcg(b, max_iters=50, tol=0.0)
    h = np.asarray(st.history)
    assert st.iters == 50
    live = ho > 1e-11
    assert np.max(np.abs(h[live] - ho[live]) / ho[live]) <= 1e-6
    assert normwise(host(x), xo) <= 1e-10


def test_fma_vcycle_and_solve_match_whole_grid_engine():
    from paper_2304_08232_gb300 import HpcgEll
    dims, levels = (32, 24, 48), 4
    n = int(np.prod(dims))
    s = _split(dims, levels)
    e = HpcgEll(*dims, levels=levels)
    r = normal(n, 94)
    zs = host(s.mg_vcycle(dev(r)))
    ze = host(e.to_natural(e.mg_vcycle(e.to_stored(dev(r)))))
    np.testing.assert_array_equal(zs, ze)  # same per-row arithmetic, halos exchanged in time
    o = OracleProblem(*dims, levels=levels)
    assert normwise(zs, o.mg(r)) <= TOL64
    b = normal(n, 95)
    xs, ss = s.pcg_solve(dev(b), max_iters=300, tol=1e-9)
    xe, se = e.pcg_solve(dev(b), max_iters=300, tol=1e-9)
    assert ss.converged and se.converged and abs(ss.iters - se.iters) <= 1
    assert normwise(host(xs), host(xe)) <= 1e-8


def test_fullsize_192cubed_vcycle_matches_whole_grid_engine():
    from paper_2304_08232_gb300 import HpcgEll
    dims = (192, 192, 192)
    n = int(np.prod(dims))
    r = normal(n, 96)
    s = _split(dims, 4)
    zs = host(s.mg_vcycle(dev(r)))
    del s
    e = HpcgEll(*dims, levels=4)
    ze = host(e.to_natural(e.mg_vcycle(e.to_stored(dev(r)))))
    np.testing.assert_array_equal(zs, ze)


def test_argument_errors():
    from paper_2304_08232_gb300 import HpcgError, HpcgSplit
    need_gpu()
    with pytest.raises(HpcgError):
        HpcgSplit(8, 8, 4, levels=3)  # nz not divisible by 2^levels
    s = HpcgSplit(8, 8, 8, levels=2)
    with pytest.raises(HpcgError):
        s.info(2, 0)
    with pytest.raises(HpcgError):
        s.info(0, 2)
    r = dev(normal(512, 97))
    with pytest.raises(HpcgError):
        s.spmv(r, out=r)
