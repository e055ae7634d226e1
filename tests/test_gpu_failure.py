"""Failure detection without a GPU fault: the persistent coarse-level kernel's
grid barriers wait a bounded number of clock cycles.  With the bound set to 0
a barrier wait runs out; the kernel records HPCG_ERR_TIMEOUT, finishes the
solve early and the host reads the status.  The context stays usable: with
the default bound restored the same handle solves correctly."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import OracleProblem
from tests.gpu_util import host, need_gpu

pytestmark = pytest.mark.gpu

HPCG_ERR_TIMEOUT = 5


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_barrier_timeout_is_reported_and_context_recovers():
    need_gpu()
    from paper_2304_08232_gb300 import HpcgProblem, _lib
    lib = _lib.load()
    g = HpcgProblem(32, 32, 32, levels=4, persistent=True)
    g.set_launch_shapes([[1, 1, 1, 1]] * 4)  # several blocks in the coarse-level kernel, so its barriers wait
    b = g.get_rhs()
    first = ctypes.c_int()
    assert lib.hpcg_persistent_levels(g.h, ctypes.byref(first)) == 0
    assert first.value >= 1  # the coarse levels run in the persistent kernel

    assert lib.hpcg_set_wait_limit(g.h, 0) == 0
    x = torch.zeros_like(b)
    st = _lib.hpcg_stats()
    rc = lib.hpcg_pcg_solve(g.h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), 10, 0.0,
                            ctypes.byref(st), _stream())
    assert rc == HPCG_ERR_TIMEOUT
    assert st.status == HPCG_ERR_TIMEOUT
    status = ctypes.c_int()
    assert lib.hpcg_device_status(g.h, ctypes.byref(status)) == 0
    assert status.value == HPCG_ERR_TIMEOUT

    # default bound back: the same handle and context solve correctly
    assert lib.hpcg_set_wait_limit(g.h, 2_000_000_000) == 0
    x2, st2 = g.pcg_solve(b, max_iters=20, tol=0.0)
    o = OracleProblem(32, 32, 32, levels=4)
    _, hr = o.pcg(o.rhs(), max_iters=20, tol=0.0)
    h = np.asarray(st2.history)
    live = hr > 1e-11
    assert np.abs(h[live] - hr[live]).max() / hr[live].min() < 1e-3
    assert np.all(np.abs(h[live] - hr[live]) / hr[live] <= 1e-6)
    assert lib.hpcg_device_status(g.h, ctypes.byref(status)) == 0 and status.value == 0


def test_vcycle_timeout_status_then_recovery():
    need_gpu()
    from paper_2304_08232_gb300 import HpcgProblem, _lib
    lib = _lib.load()
    g = HpcgProblem(16, 16, 16, levels=4, precision="mixed", persistent=True)
    # one line per block: the coarse-level kernel then has more than one block,
    # so its grid barriers wait (a single block never waits, whatever the limit)
    g.set_launch_shapes([[1, 1, 1, 1]] * 4)
    r = torch.ones(16 ** 3, dtype=torch.float64, device="cuda")
    first = ctypes.c_int()
    assert lib.hpcg_persistent_levels(g.h, ctypes.byref(first)) == 0 and first.value >= 1
    assert lib.hpcg_set_wait_limit(g.h, 0) == 0
    g.mg_vcycle(r)
    status = ctypes.c_int()
    assert lib.hpcg_device_status(g.h, ctypes.byref(status)) == 0 and status.value == HPCG_ERR_TIMEOUT
    assert lib.hpcg_set_wait_limit(g.h, 2_000_000_000) == 0
    z = host(g.mg_vcycle(r))
    assert lib.hpcg_device_status(g.h, ctypes.byref(status)) == 0 and status.value == 0
    zr = OracleProblem(16, 16, 16, levels=4).mg(np.ones(16 ** 3))
    assert np.abs(z - zr).max() / np.abs(zr).max() < 2e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("dims", [(32, 32, 32), (16, 24, 40), (64, 48, 32)])
def test_persistent_coarse_kernel_is_bit_identical(dims, precision):
    """The persistent coarse-level kernel runs the same arithmetic as one
    launch per step: V-cycles and CG histories agree bit for bit."""
    need_gpu()
    from hpcg_inputs import normal
    from paper_2304_08232_gb300 import HpcgProblem, _lib
    lib = _lib.load()
    # the persistent kernel keeps z in FP64: compare the two in that form
    gp = HpcgProblem(*dims, levels=4, precision=precision, persistent=True, block_fp=False)
    gs = HpcgProblem(*dims, levels=4, precision=precision, persistent=False, block_fp=False)
    first = ctypes.c_int()
    lib.hpcg_persistent_levels(gp.h, ctypes.byref(first))
    assert 1 <= first.value <= 3
    # same launch shapes for both (the shape never changes the arithmetic, but
    # the comparison is clearer with identical launches on the per-step levels)
    shapes = gp.autotune()
    gs.set_launch_shapes(shapes)
    n = int(np.prod(dims))
    r = torch.as_tensor(normal(n, 11), device="cuda")
    np.testing.assert_array_equal(host(gp.mg_vcycle(r)), host(gs.mg_vcycle(r)))
    b = gp.get_rhs()
    xp, stp = gp.pcg_solve(b, max_iters=15, tol=0.0)
    xs, sts = gs.pcg_solve(b, max_iters=15, tol=0.0)
    np.testing.assert_array_equal(np.asarray(stp.history), np.asarray(sts.history))
    np.testing.assert_array_equal(host(xp), host(xs))
