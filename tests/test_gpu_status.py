"""Status paths of the C ABI on the GPU: CG breakdown on a negative definite
operator and on a non-finite right-hand side, the not-converged status, a
breakdown confined to one grid of a batch, and argument errors; after each,
the same handle still computes what the oracle computes."""
import ctypes

import numpy as np
import pytest
import torch

from hpcg_inputs import normal
from oracle import OracleProblem
from tests.gpu_util import TOL64, dev, host, need_gpu, normwise

pytestmark = pytest.mark.gpu

OK, INVALID_ARG, BREAKDOWN, NOT_CONVERGED, NO_WORKSPACE, UNSUPPORTED = 0, 1, 3, 4, 6, 8


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _raw_solve(g, b, x, max_iters, tol):
    from paper_2304_08232_gb300.binding import _new_stats, _Stats
    st, hist = _new_stats(max(max_iters, 1))
    rc = g.lib.hpcg_pcg_solve(g.h, _p(b), _p(x), max_iters, tol, ctypes.byref(st), _s())
    torch.cuda.synchronize()
    return rc, _Stats(st, hist)


def _history_close(h, h_ref):
    h, h_ref = np.asarray(h), np.asarray(h_ref)
    assert len(h) == len(h_ref)
    assert np.max(np.abs(h - h_ref) / h_ref) <= 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_negative_definite_operator_breaks_down_then_recovers(precision):
    """kappa = -60 makes every eigenvalue of A negative (the 27-point part lies
    in (0, 54)): p.Ap < 0 at the first iteration, which CG cannot take."""
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    dims = (16, 16, 16)
    n = int(np.prod(dims))
    g = HpcgProblem(*dims, levels=3, precision=precision)
    g.set_kappa(torch.full((n,), -60.0, dtype=torch.float64, device="cuda"))
    b = dev(normal(n, 5))
    x = torch.zeros_like(b)
    rc, st = _raw_solve(g, b, x, 20, 1e-8)
    assert rc == BREAKDOWN and st.status == BREAKDOWN
    assert st.iters == 0 and not st.converged
    assert torch.all(x == 0)
    # the same handle, with the operator restored, solves as the oracle does
    g.set_kappa(torch.zeros(n, dtype=torch.float64, device="cuda"))
    x.zero_()
    o = OracleProblem(*dims, levels=3)
    if precision == "fp64":
        rc, st = _raw_solve(g, b, x, 10, 0.0)
        assert rc == OK and st.iters == 10
        xr, hr = o.pcg(host(b), max_iters=10, tol=0.0)
        _history_close(st.history, hr)
        assert normwise(host(x), xr) <= 1e-10
    else:
        rc, st = _raw_solve(g, b, x, 200, 1e-9)
        assert rc == OK and st.converged
        bh = host(b)
        assert np.linalg.norm(bh - o.spmv(host(x))) / np.linalg.norm(bh) <= 2e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nonfinite_rhs_breaks_down_at_start(precision):
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    dims = (16, 16, 16)
    n = int(np.prod(dims))
    g = HpcgProblem(*dims, levels=4, precision=precision)
    bh = normal(n, 6)
    for bad in (np.nan, np.inf):
        b = bh.copy()
        b[777] = bad
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        rc, st = _raw_solve(g, dev(b), x, 20, 1e-8)
        assert rc == BREAKDOWN and st.status == BREAKDOWN and st.iters == 0
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc, st = _raw_solve(g, dev(bh), x, 200, 1e-9)
    assert rc == OK and st.converged


def test_not_converged_status_and_history():
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    dims = (16, 16, 16)
    n = int(np.prod(dims))
    g = HpcgProblem(*dims, levels=4)
    b = normal(n, 7)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc, st = _raw_solve(g, dev(b), x, 3, 1e-30)
    assert rc == NOT_CONVERGED and st.status == NOT_CONVERGED
    assert st.iters == 3 and not st.converged
    xr, hr = OracleProblem(*dims, levels=4).pcg(b, max_iters=3, tol=1e-30)
    _history_close(st.history, hr)
    assert abs(st.rel_res - hr[-1]) <= 1e-6 * hr[-1]
    # max_iters = 0 runs nothing and reports the initial residual
    x.zero_()
    rc, st = _raw_solve(g, dev(b), x, 0, 0.0)
    assert rc == OK and st.iters == 0 and torch.all(x == 0)


def test_breakdown_of_one_batch_grid_leaves_the_others():
    from paper_2304_08232_gb300 import HpcgBatch
    from paper_2304_08232_gb300.binding import _new_stats, _Stats
    from paper_2304_08232_gb300._lib import hpcg_stats
    need_gpu()
    dims = [(16, 16, 16), (32, 16, 16), (16, 32, 24)]
    g = HpcgBatch(dims, levels=3)
    b = normal(g.n, 8)
    b[g.offsets[1] + 100] = np.nan
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    sts = (hpcg_stats * 3)()
    hists = []
    for k in range(3):
        st, hist = _new_stats(100)
        sts[k] = st
        hists.append(hist)
    rc = g.lib.hpcg_pcg_solve_batch(g.h, _p(dev(b)), _p(x), 100, 1e-9, sts, _s())
    torch.cuda.synchronize()
    stats = [_Stats(sts[k], hists[k]) for k in range(3)]
    assert rc == BREAKDOWN
    assert stats[1].status == BREAKDOWN and stats[1].iters == 0
    xh = host(x)
    for k in (0, 2):
        s = slice(g.offsets[k], g.offsets[k + 1])
        o = OracleProblem(*dims[k], levels=3)
        xr, hr = o.pcg(b[s], max_iters=100, tol=1e-9)
        assert stats[k].status == OK and stats[k].converged and stats[k].iters == len(hr)
        _history_close(stats[k].history, hr)
        assert normwise(xh[s], xr) <= 1e-8


def test_argument_errors_leave_the_handle_usable():
    from paper_2304_08232_gb300 import HpcgBatch, HpcgProblem
    need_gpu()
    dims = (16, 16, 16)
    n = int(np.prod(dims))
    g = HpcgProblem(*dims, levels=4)
    lib, h, s = g.lib, g.h, _s()
    a = dev(normal(n, 9))
    c = torch.zeros_like(a)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert lib.hpcg_spmv(h, 4, _p(a), _p(c), s) == INVALID_ARG           # level out of range
    assert lib.hpcg_spmv(h, 0, None, _p(c), s) == INVALID_ARG            # null vector
    assert lib.hpcg_rbgs_color(h, 0, 8, _p(a), _p(c), s) == INVALID_ARG  # colour out of range
    assert lib.hpcg_restrict_residual(h, 3, _p(a), _p(c), _p(c), s) == INVALID_ARG  # no coarser level
    assert lib.hpcg_mg_vcycle(h, _p(a), _p(a), s) == INVALID_ARG          # r and z alias
    assert lib.hpcg_dot(h, -1, _p(a), _p(a), _p(out), s) == INVALID_ARG
    assert lib.hpcg_pcg_solve(h, _p(a), _p(c), 8193, 0.0, None, s) == INVALID_ARG
    assert lib.hpcg_pcg_solve(h, _p(a), _p(c), -1, 0.0, None, s) == INVALID_ARG
    assert lib.hpcg_pcg_solve_multi(h, 2, _p(a), _p(c), 5, 0.0, None, s) == NO_WORKSPACE  # max_rhs = 0
    assert lib.hpcg_pcg_backward(h, _p(a), _p(c), _p(a), None, 5, 0.0, None, s) == INVALID_ARG  # grad_b aliases x
    assert lib.hpcg_pcg_solve_batch(h, _p(a), _p(c), 5, 0.0, None, s) == UNSUPPORTED
    bad = (ctypes.c_int * 16)(*([4, 4, 4, 4] * 3 + [4, 4, 0, 4]))
    assert lib.hpcg_set_launch_shapes(h, bad) == INVALID_ARG
    assert lib.hpcg_set_wait_limit(h, -1) == INVALID_ARG
    nb = ctypes.c_size_t()
    assert lib.hpcg_workspace_bytes(h, ctypes.byref(nb)) == OK
    ws = torch.empty(nb.value + 512, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) & ~255
    assert lib.hpcg_bind_workspace(h, ctypes.c_void_p(base), nb.value - 8) == NO_WORKSPACE
    assert lib.hpcg_bind_workspace(h, ctypes.c_void_p(base + 8), nb.value) == INVALID_ARG
    bt = HpcgBatch([(16, 16, 16)], levels=2)
    assert bt.lib.hpcg_set_kappa(bt.h, _p(a), s) == UNSUPPORTED
    st = ctypes.c_int(-1)
    assert lib.hpcg_device_status(h, ctypes.byref(st)) == OK and st.value == OK
    # the handle is unchanged by all of the above
    o = OracleProblem(*dims, levels=4)
    assert normwise(host(g.spmv(a)), o.spmv(host(a))) <= TOL64
    x, stt = g.pcg_solve(g.get_rhs(), max_iters=5, tol=0.0)
    _, hr = o.pcg(o.rhs(), max_iters=5, tol=0.0)
    _history_close(stt.history, hr)
