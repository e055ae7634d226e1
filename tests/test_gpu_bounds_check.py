"""The bounds-checking build (-DHPCG_BOUNDS_CHECK; compute-sanitizer is not
available on the GPU pool): every index range the default FP64 path touches
(colour-pair runs in block floating point with the fused restriction and
refinement, the staged SpMV, the CG updates, dot products and reductions, the
level-vector conversions) is checked against its array's extent, a miss
counted and skipped.  Tiny, ragged and odd-sized grids, a kappa field, the
stage calls, mixed precision and a batch of uneven grids run through it; no
range may be missed, and the checked library computes the same bits as the
normal one (in range, the checks skip nothing)."""
import ctypes

import numpy as np
import pytest
import torch

from hpcg_inputs import normal, uniform
from tests.gpu_util import dev, host, need_gpu

pytestmark = pytest.mark.gpu

GRIDS = [((2, 2, 2), 1), ((3, 5, 7), 1), ((4, 6, 10), 2), ((6, 10, 14), 2), ((34, 6, 10), 2), ((24, 8, 16), 3),
         ((16, 16, 16), 4), ((64, 32, 48), 4), ((96, 64, 80), 4)]


@pytest.fixture(scope="module")
def libs():
    need_gpu()
    from paper_2304_08232_gb300 import _lib
    chk = _lib.load_checked()
    cnt, first = ctypes.c_longlong(), (ctypes.c_longlong * 2)()
    assert chk.hpcg_bounds_status(ctypes.byref(cnt), first, 1) == 0
    assert _lib.load().hpcg_bounds_status(ctypes.byref(cnt), first, 0) == 8  # the normal build has no checks
    return _lib.load(), chk


def _violations(chk, reset=True):
    torch.cuda.synchronize()
    cnt, first = ctypes.c_longlong(), (ctypes.c_longlong * 2)()
    assert chk.hpcg_bounds_status(ctypes.byref(cnt), first, 1 if reset else 0) == 0
    return cnt.value, (first[0], first[1])


@pytest.mark.parametrize("dims,levels", GRIDS)
@pytest.mark.parametrize("with_kappa", [False, True])
def test_default_path_stays_in_bounds(libs, dims, levels, with_kappa):
    from paper_2304_08232_gb300 import HpcgProblem
    normal_lib, chk = libs
    n = int(np.prod(dims))
    kappa = dev(uniform(n, 0.0, 1.0, 401)) if with_kappa else None
    gc = HpcgProblem(*dims, levels=levels, kappa=kappa, lib=chk)
    gn = HpcgProblem(*dims, levels=levels, kappa=kappa, lib=normal_lib)
    gn.set_launch_shapes(gc.autotune())
    r = dev(normal(n, 402))
    for l in range(levels):
        x = dev(normal(gc.level_n(l), 403 + l))
        np.testing.assert_array_equal(host(gc.spmv(x, level=l)), host(gn.spmv(x, level=l)))
    np.testing.assert_array_equal(host(gc.mg_vcycle(r)), host(gn.mg_vcycle(r)))
    b = gc.get_rhs()
    xc, sc = gc.pcg_solve(b, max_iters=6, tol=0.0)
    xn, sn = gn.pcg_solve(b, max_iters=6, tol=0.0)
    np.testing.assert_array_equal(host(xc), host(xn))
    z = torch.zeros_like(r)
    for l in range(levels):
        gc.mg_stage(l, "pre", r, z)
    for l in range(levels - 2, -1, -1):
        gc.mg_stage(l, "refine", r, z)
        gc.mg_stage(l, "post", r, z)
    for l in range(1, levels):
        rl, zl = gc.get_level_vectors(l)
        gc.set_level_vectors(l, r=rl, z=zl)
    assert _violations(chk) == (0, (-1, -1))


@pytest.mark.parametrize("dims,levels", [((16, 16, 16), 4), ((48, 32, 24), 3), ((6, 10, 14), 2)])
def test_mixed_precision_and_fp64_storage_stay_in_bounds(libs, dims, levels):
    from paper_2304_08232_gb300 import HpcgProblem
    _, chk = libs
    n = int(np.prod(dims))
    b = dev(normal(n, 404))
    for kw in ({"precision": "mixed"}, {"block_fp": False}, {"persistent": True}):
        g = HpcgProblem(*dims, levels=levels, lib=chk, **kw)
        g.pcg_solve(b, max_iters=5, tol=0.0)
        g.mg_vcycle(b)
    assert _violations(chk) == (0, (-1, -1))


def test_uneven_batch_stays_in_bounds(libs):
    from paper_2304_08232_gb300 import HpcgBatch
    normal_lib, chk = libs
    dims = [(32, 48, 16), (16, 16, 16), (64, 32, 32), (48, 16, 80), (96, 32, 16)]
    bc = HpcgBatch(dims, levels=4, lib=chk)
    bn = HpcgBatch(dims, levels=4, lib=normal_lib)
    b = dev(normal(bc.n, 405))
    xc, _ = bc.pcg_solve(b, max_iters=12, tol=1e-8)
    xn, _ = bn.pcg_solve(b, max_iters=12, tol=1e-8)
    assert _violations(chk) == (0, (-1, -1))
    assert np.max(np.abs(host(xc) - host(xn))) <= 1e-12 * np.max(np.abs(host(xn)))
