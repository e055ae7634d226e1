"""The FP64 V-cycle with z in block floating point (hpcg_options.block_fp, the
default) against the V-cycle that keeps z in FP64 and against the oracle:
agreement with and without kappa, CG histories, dynamic range, NaN
propagation, and the FP64 path taken for vectors that are not 16-byte
aligned."""
import numpy as np
import pytest
import torch

from hpcg_inputs import normal, uniform
from oracle import OracleProblem
from tests.gpu_util import TOL64, dev, host, need_gpu, normwise

pytestmark = pytest.mark.gpu

CASES = [((16, 16, 16), 4), ((64, 32, 48), 4), ((8, 12, 16), 2), ((2, 2, 2), 1), ((96, 64, 80), 4), ((384, 16, 16), 3)]


def _pair(dims, levels, kappa=None):
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    k = None if kappa is None else dev(kappa)
    return (HpcgProblem(*dims, levels=levels, kappa=k), HpcgProblem(*dims, levels=levels, kappa=k, block_fp=False))


@pytest.mark.parametrize("dims,levels", CASES)
@pytest.mark.parametrize("with_kappa", [False, True])
def test_block_fp_vcycle_matches_fp64_and_oracle(dims, levels, with_kappa):
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 4) if with_kappa else None
    gb, gf = _pair(dims, levels, kappa)
    o = OracleProblem(*dims, levels=levels, kappa=kappa)
    r = normal(n, 31)
    zb, zf, zo = host(gb.mg_vcycle(dev(r))), host(gf.mg_vcycle(dev(r))), o.mg(r)
    assert normwise(zb, zo) <= TOL64
    assert normwise(zb, zf) <= TOL64
    if n >= 4096:  # a different arithmetic ran (same values to rounding, not the same bits)
        assert not np.array_equal(zb, zf)


@pytest.mark.parametrize("with_kappa", [False, True])
def test_block_fp_cg_history(with_kappa):
    dims, levels = (32, 48, 40), 4
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 5) if with_kappa else None
    gb, gf = _pair(dims, levels, kappa)
    o = OracleProblem(*dims, levels=levels, kappa=kappa)
    b = normal(n, 32)
    xb, sb = gb.pcg_solve(dev(b), max_iters=40, tol=0.0)
    xf, sf = gf.pcg_solve(dev(b), max_iters=40, tol=0.0)
    xo, ho = o.pcg(b, max_iters=40, tol=0.0)
    for h in (sb.history, sf.history):
        live = ho > 1e-11
        assert np.max(np.abs(np.asarray(h)[live] - ho[live]) / ho[live]) <= 1e-6
    assert normwise(host(xb), xo) <= 1e-10


@pytest.mark.parametrize("scale", [1e-280, 1e-150, 1.0, 1e150, 1e280])
def test_block_fp_dynamic_range(scale):
    """Uniform scaling of r by powers far from 1, and values spread over 40
    decades within every line: the line exponents follow the data."""
    dims, levels = (32, 32, 32), 4
    n = int(np.prod(dims))
    gb, _ = _pair(dims, levels)
    o = OracleProblem(*dims, levels=levels)
    r = normal(n, 33) * scale
    assert normwise(host(gb.mg_vcycle(dev(r))), o.mg(r)) <= TOL64
    spread = normal(n, 34) * 10.0 ** np.random.default_rng(35).uniform(-20, 20, n)
    assert normwise(host(gb.mg_vcycle(dev(spread))), o.mg(spread)) <= TOL64


def test_block_fp_nan_propagates_and_clears():
    dims, levels = (32, 32, 32), 4
    n = int(np.prod(dims))
    gb, _ = _pair(dims, levels)
    o = OracleProblem(*dims, levels=levels)
    r = normal(n, 36)
    bad = r.copy()
    bad[5000] = np.nan
    assert np.isnan(host(gb.mg_vcycle(dev(bad)))).any()
    assert normwise(host(gb.mg_vcycle(dev(r))), o.mg(r)) <= TOL64  # no NaN left behind in the levels


def test_unaligned_vectors_take_the_fp64_path():
    dims, levels = (32, 32, 32), 4
    n = int(np.prod(dims))
    gb, _ = _pair(dims, levels)
    o = OracleProblem(*dims, levels=levels)
    r = normal(n, 37)
    rb = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    zb = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    rb[1:] = dev(r)
    gb.mg_vcycle(rb[1:], out=zb[1:])  # 8-byte offsets
    assert normwise(host(zb[1:]), o.mg(r)) <= TOL64


@pytest.mark.parametrize("dims", [(64, 48, 32), (96, 96, 96), (32, 32, 64)])
def test_cluster_tail_is_bit_identical(dims):
    """The coarse levels in one cluster launch compute the same bits as one
    launch per run (hpcg_options.cluster_tail)."""
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    n = int(np.prod(dims))
    gt = HpcgProblem(*dims, levels=4, cluster_tail=True)
    gs = HpcgProblem(*dims, levels=4, cluster_tail=False)
    gs.set_launch_shapes(gt.autotune())
    r = dev(normal(n, 38))
    np.testing.assert_array_equal(host(gt.mg_vcycle(r)), host(gs.mg_vcycle(r)))
    b = gt.get_rhs()
    xt, st = gt.pcg_solve(b, max_iters=12, tol=0.0)
    xs, ss = gs.pcg_solve(b, max_iters=12, tol=0.0)
    np.testing.assert_array_equal(np.asarray(st.history), np.asarray(ss.history))
    np.testing.assert_array_equal(host(xt), host(xs))
    # and the profile shows the cluster kernel in place of the coarse runs
    pr = gt.profile_iteration(b)
    assert pr["persistent_coarse_ms"] > 0 and pr["smoother_ms"][3] == 0


def test_cluster_tail_with_kappa_matches_oracle():
    dims = (48, 32, 64)
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 39)
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    g = HpcgProblem(*dims, levels=4, kappa=dev(kappa), cluster_tail=True)
    o = OracleProblem(*dims, levels=4, kappa=kappa)
    r = normal(n, 40)
    assert normwise(host(g.mg_vcycle(dev(r))), o.mg(r)) <= TOL64


SPLIT_CASES = [((96, 64, 80), 4), ((192, 32, 48), 4), ((256, 16, 32), 3), ((128, 40, 24), 4)]


@pytest.mark.parametrize("dims,levels", SPLIT_CASES)
@pytest.mark.parametrize("with_kappa", [False, True])
def test_split_lines_give_the_same_vcycle_bits(dims, levels, with_kappa):
    """hpcg_options.bfp_split: lines of 2-4 chunks with one warp per chunk give
    the V-cycle of one warp per line bit for bit, for any launch shape."""
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    n = int(np.prod(dims))
    kappa = dev(uniform(n, 0.0, 1.0, 42)) if with_kappa else None
    g1 = HpcgProblem(*dims, levels=levels, kappa=kappa)
    gs = HpcgProblem(*dims, levels=levels, kappa=kappa, bfp_split=True)
    r = dev(normal(n, 43))
    z1 = host(g1.mg_vcycle(r))
    np.testing.assert_array_equal(host(gs.mg_vcycle(r)), z1)
    for lpc, zc in [(1, 1), (8, 4), (2, 3)]:
        gs.set_launch_shapes([[1, 1, lpc, zc]] * levels)
        np.testing.assert_array_equal(host(gs.mg_vcycle(r)), z1)


@pytest.mark.parametrize("dims,levels", SPLIT_CASES[:2])
def test_split_lines_cg_matches_oracle(dims, levels):
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    n = int(np.prod(dims))
    gs = HpcgProblem(*dims, levels=levels, bfp_split=True)
    o = OracleProblem(*dims, levels=levels)
    b = normal(n, 44)
    x, st = gs.pcg_solve(dev(b), max_iters=30, tol=0.0)
    xo, ho = o.pcg(b, max_iters=30, tol=0.0)
    h = np.asarray(st.history)
    live = ho > 1e-11
    assert np.max(np.abs(h[live] - ho[live]) / ho[live]) <= 1e-6
    assert normwise(host(x), xo) <= 1e-10
