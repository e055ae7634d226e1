"""GPU parity of the batched forms: many right-hand sides on one grid
(hpcg_pcg_solve_multi) and a batch of independent grids of uneven size
(hpcg_setup_batch / hpcg_pcg_solve_batch), each system checked against the
CPU oracle solving it alone."""
import numpy as np
import pytest
import torch

from hpcg_inputs import multi_rhs, normal, uneven_batch_dims
from oracle import OracleProblem
from tests.gpu_util import dev, host, need_gpu, normwise

pytestmark = pytest.mark.gpu


def _history_close(h, h_ref, floor=1e-11):
    h, h_ref = np.asarray(h), np.asarray(h_ref)
    assert len(h) == len(h_ref), (len(h), len(h_ref))
    live = h_ref > floor
    rel = np.abs(h[live] - h_ref[live]) / h_ref[live]
    assert rel.max() <= 1e-6, rel


@pytest.mark.parametrize("nrhs", [1, 3, 8, 32])
def test_multi_rhs_fixed_iterations(nrhs):
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    dims, levels = (16, 16, 24), 3
    n = int(np.prod(dims))
    g = HpcgProblem(*dims, levels=levels, max_rhs=nrhs)
    o = OracleProblem(*dims, levels=levels)
    B = multi_rhs(n, nrhs, seed=2)
    X, sts = g.pcg_solve_multi(dev(B), max_iters=20, tol=0.0)
    Xh = host(X)
    for k in range(nrhs):
        xr, hr = o.pcg(B[k], max_iters=20, tol=0.0)
        assert sts[k].iters == 20
        _history_close(sts[k].history, hr)
        assert normwise(Xh[k], xr) <= 1e-9


def test_multi_rhs_each_stops_on_its_own():
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    dims, levels = (16, 24, 16), 3
    n = int(np.prod(dims))
    g = HpcgProblem(*dims, levels=levels, max_rhs=4)
    o = OracleProblem(*dims, levels=levels)
    B = multi_rhs(n, 4, seed=5)
    B[1] *= 1e-3                          # scaling does not change the relative history
    B[2] = o.rhs()                        # smooth right-hand side converges at another pace
    X0 = np.zeros((4, n))
    X0[3] = normal(n, 9)                  # non-zero initial guess
    X, sts = g.pcg_solve_multi(dev(B), X0=dev(X0), max_iters=200, tol=1e-9)
    Xh = host(X)
    for k in range(4):
        xr, hr = o.pcg(B[k], x0=X0[k], max_iters=200, tol=1e-9)
        assert sts[k].converged and sts[k].iters == len(hr)
        _history_close(sts[k].history, hr)
        assert normwise(Xh[k], xr) <= 1e-7


def test_uneven_batch_against_oracle():
    from paper_2304_08232_gb300 import HpcgBatch
    need_gpu()
    dims = [(16, 16, 16), (32, 8, 16), (8, 24, 16), (8, 8, 8), (24, 16, 32)]
    levels = 3
    bat = HpcgBatch(dims, levels=levels)
    offs = bat.offsets
    b = normal(bat.n, 7)
    x, sts = bat.pcg_solve(dev(b), max_iters=200, tol=1e-9)
    xh = host(x)
    for i, d in enumerate(dims):
        o = OracleProblem(*d, levels=levels)
        bi = b[offs[i]:offs[i + 1]]
        xr, hr = o.pcg(bi, max_iters=200, tol=1e-9)
        assert sts[i].converged and sts[i].iters == len(hr), (i, sts[i], len(hr))
        _history_close(sts[i].history, hr)
        assert normwise(xh[offs[i]:offs[i + 1]], xr) <= 1e-7


def test_uneven_batch_fixed_iterations_mixed_precision():
    from paper_2304_08232_gb300 import HpcgBatch
    need_gpu()
    dims = [(16, 16, 16), (32, 16, 8), (16, 8, 24)]
    bat = HpcgBatch(dims, levels=3, precision="mixed")
    b = normal(bat.n, 8)
    x, sts = bat.pcg_solve(dev(b), max_iters=200, tol=1e-9)
    xh = host(x)
    for i, d in enumerate(dims):
        o = OracleProblem(*d, levels=3)
        bi = b[bat.offsets[i]:bat.offsets[i + 1]]
        xi = xh[bat.offsets[i]:bat.offsets[i + 1]]
        assert sts[i].converged
        assert np.linalg.norm(bi - o.spmv(xi)) / np.linalg.norm(bi) <= 2e-9


def test_full_uneven_batch_64_grids():
    """The 64-grid workload: edges from {32,48,64,80,96} (seed 3), 4 levels, to 1e-8."""
    from paper_2304_08232_gb300 import HpcgBatch, HpcgProblem
    need_gpu()
    dims = [tuple(int(v) for v in d) for d in uneven_batch_dims(64, seed=3)]
    bat = HpcgBatch(dims, levels=4)
    b = dev(normal(bat.n, 3))
    x, sts = bat.pcg_solve(b, max_iters=500, tol=1e-8)
    assert all(s.converged for s in sts)
    # true residual of every instance with the (parity-tested) single-grid SpMV
    for i, d in enumerate(dims):
        lo, hi = bat.offsets[i], bat.offsets[i + 1]
        g = HpcgProblem(*d, levels=1)
        r = b[lo:hi] - g.spmv(x[lo:hi].contiguous())
        rel = float(torch.linalg.norm(r) / torch.linalg.norm(b[lo:hi]))
        assert rel <= 1.01e-8, (i, d, rel)
    # two instances against the oracle
    for i in (0, 63):
        lo, hi = bat.offsets[i], bat.offsets[i + 1]
        o = OracleProblem(*dims[i], levels=4)
        xr, hr = o.pcg(host(b[lo:hi]), max_iters=500, tol=1e-8)
        assert sts[i].iters == len(hr)


def test_full_multi_rhs_32_on_128cubed():
    """32 right-hand sides ~ N(0,1) (seed 2) on 128^3, to 1e-8."""
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    n = 128 ** 3
    g = HpcgProblem(128, 128, 128, levels=4, max_rhs=32)
    B = dev(multi_rhs(n, 32, seed=2))
    X, sts = g.pcg_solve_multi(B, max_iters=500, tol=1e-8)
    assert all(s.converged for s in sts)
    for k in (0, 17, 31):
        r = B[k] - g.spmv(X[k].contiguous())
        assert float(torch.linalg.norm(r) / torch.linalg.norm(B[k])) <= 1.01e-8
    # one right-hand side against the single-RHS solver
    x0, st0 = g.pcg_solve(B[5].contiguous(), max_iters=500, tol=1e-8)
    assert st0.iters == sts[5].iters
    assert normwise(host(X[5]), host(x0)) <= 1e-9
