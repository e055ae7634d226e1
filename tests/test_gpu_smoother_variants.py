"""Smoother variants on the GPU against the oracle: the forward-only sweep
(the ablation of the symmetric reading) and several smoother applications
per level (pre_sweeps, post_sweeps), whose V-cycle is composed here from the
oracle's own steps (smoother, residual, injection, refinement) in Listing 1's
order."""
import numpy as np
import pytest

from hpcg_inputs import normal
from oracle import OracleProblem
from tests.gpu_util import TOL64, dev, host, need_gpu, normwise

pytestmark = pytest.mark.gpu


def _mg_composed(o, r, l, pre, post, levels):
    """Listing 1 with `pre` and `post` smoother applications (one on the
    coarsest level), from the oracle's steps."""
    z = np.zeros(o.n(l))
    sweeps = 1 if l == levels - 1 else pre
    for _ in range(sweeps):
        z = o.rbgs(r, z, l)
    if l == levels - 1:
        return z
    rc = o.restrict(r - o.spmv(z, l), l)
    zc = _mg_composed(o, rc, l + 1, pre, post, levels)
    z = o.prolong_add(zc, z, l)
    for _ in range(post):
        z = o.rbgs(r, z, l)
    return z


@pytest.mark.parametrize("dims,levels", [((16, 16, 16), 4), ((32, 24, 16), 3), ((8, 12, 16), 2)])
def test_forward_only_vcycle_and_pcg(dims, levels):
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    n = int(np.prod(dims))
    g = HpcgProblem(*dims, levels=levels, symmetric=False)
    o = OracleProblem(*dims, levels=levels, symmetric=False)
    r = normal(n, 47)
    assert normwise(host(g.mg_vcycle(dev(r))), o.mg(r)) <= TOL64
    b = normal(n, 48)
    x, st = g.pcg_solve(dev(b), max_iters=20, tol=0.0)
    xr, hr = o.pcg(b, max_iters=20, tol=0.0)
    live = hr > 1e-11
    assert np.max(np.abs(np.asarray(st.history)[live] - hr[live]) / hr[live]) <= 1e-6


@pytest.mark.parametrize("pre,post", [(2, 2), (1, 3), (3, 1)])
@pytest.mark.parametrize("block_fp", [True, False])
def test_several_smoother_applications(pre, post, block_fp):
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    dims, levels = (32, 16, 24), 3
    n = int(np.prod(dims))
    g = HpcgProblem(*dims, levels=levels, pre_sweeps=pre, post_sweeps=post, block_fp=block_fp)
    o = OracleProblem(*dims, levels=levels)
    r = normal(n, 49)
    assert normwise(host(g.mg_vcycle(dev(r))), _mg_composed(o, r, 0, pre, post, levels)) <= TOL64
