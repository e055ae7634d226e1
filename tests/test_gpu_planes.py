"""The colour-pair runs of one plane parity in one launch (hpcg_options.
fuse_planes, k_gs_planes_bfp) against one launch per run: the same bits for
the V-cycle, the CG solve and every stage of hpcg_mg_stage, with and without
kappa, on grids with odd line counts, several chunks per line and two
smoother sweeps (groups of three runs and more groups), and against the
oracle (Listing 1, Section II-C)."""
import numpy as np
import pytest

from hpcg_inputs import normal, uniform
from oracle import OracleProblem
from tests.gpu_util import TOL64, dev, host, need_gpu, normwise
from tests.test_gpu_smoother_variants import _mg_composed

pytestmark = pytest.mark.gpu

CASES = [((16, 16, 16), 4), ((64, 32, 48), 4), ((34, 18, 66), 2), ((96, 64, 80), 4), ((192, 24, 40), 3), ((256, 16, 32), 3)]


def _pair(dims, levels, kappa=None, **kw):
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    k = None if kappa is None else dev(kappa)
    gf = HpcgProblem(*dims, levels=levels, kappa=k, fuse_planes=1, **kw)
    gs = HpcgProblem(*dims, levels=levels, kappa=k, fuse_planes=-1, **kw)
    gs.set_launch_shapes(gf.autotune())
    return gf, gs


@pytest.mark.parametrize("dims,levels", CASES)
@pytest.mark.parametrize("with_kappa", [False, True])
def test_planes_bit_identical_vcycle_and_solve(dims, levels, with_kappa):
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 51) if with_kappa else None
    gf, gs = _pair(dims, levels, kappa)
    r = dev(normal(n, 52))
    zf = host(gf.mg_vcycle(r))
    np.testing.assert_array_equal(zf, host(gs.mg_vcycle(r)))
    assert normwise(zf, OracleProblem(*dims, levels=levels, kappa=kappa).mg(host(r))) <= TOL64
    b = gf.get_rhs()
    xf, sf = gf.pcg_solve(b, max_iters=15, tol=0.0)
    xs, ss = gs.pcg_solve(b, max_iters=15, tol=0.0)
    np.testing.assert_array_equal(np.asarray(sf.history), np.asarray(ss.history))
    np.testing.assert_array_equal(host(xf), host(xs))


@pytest.mark.parametrize("dims,levels", [((32, 16, 24), 3), ((64, 32, 48), 4)])
def test_planes_two_sweeps(dims, levels):
    """pre- and post-smoothing by two symmetric sweeps: runs of one class meet
    across the sweeps, and groups are cut at three runs."""
    n = int(np.prod(dims))
    gf, gs = _pair(dims, levels, pre_sweeps=2, post_sweeps=2)
    r = dev(normal(n, 53))
    zf = host(gf.mg_vcycle(r))
    np.testing.assert_array_equal(zf, host(gs.mg_vcycle(r)))
    assert normwise(zf, _mg_composed(OracleProblem(*dims, levels=levels), host(r), 0, 2, 2, levels)) <= TOL64


def _levels_state(g, l, levels):
    """z_l (and r_l above the finest level), r_{l+1} and z_{l+1} as host arrays."""
    out = []
    for k in (l, l + 1):
        if k < levels:
            rk, zk = g.get_level_vectors(k, r=k > 0)
            out += [host(zk)] + ([host(rk)] if k > 0 else [])
    return out


def _set_levels(g, src, l, levels):
    for k in (l, l + 1):
        if k < levels:
            rk, zk = src.get_level_vectors(k, r=k > 0)
            g.set_level_vectors(k, rk if k > 0 else None, zk)


@pytest.mark.parametrize("dims,levels", [((64, 32, 48), 4), ((96, 64, 80), 4)])
def test_planes_stages_bit_identical(dims, levels):
    """Each stage of each level (pre-smoothing with its restriction, the
    refinement alone, refinement + post-smoothing), started from the same
    level vectors, leaves the same bits either way."""
    import torch
    n = int(np.prod(dims))
    gf, gs = _pair(dims, levels)
    r0 = dev(normal(n, 54))
    gf.mg_vcycle(r0)  # level vectors from one V-cycle to start the stages from
    for l in range(levels):
        for stage in ("pre", "refine", "post"):
            if l == levels - 1 and stage != "pre":
                continue
            states = []
            for g in (gs, gf):  # gs first: gf's vectors are the common start
                _set_levels(g, gf, l, levels)
                g.mg_stage(l, stage, r0, torch.zeros_like(r0))
                states.append(_levels_state(g, l, levels))
            for a, b in zip(states[0], states[1]):
                np.testing.assert_array_equal(a, b)


def test_planes_full_size_vcycle():
    n = 192 ** 3
    gf, gs = _pair((192, 192, 192), 4)
    r = dev(normal(n, 55))
    np.testing.assert_array_equal(host(gf.mg_vcycle(r)), host(gs.mg_vcycle(r)))
