"""The staged SpMV (each plane's x-lines copied into shared memory two planes
ahead and converted to fixed point once per block, hpcg_spmv.cuh): the paths
it adds beside the parity tests of test_gpu_steps.py.  Input that is not
16-byte aligned (8-byte copies) gives the same bits as aligned input; huge and
non-finite values make a block finish with FP64 sums (NaN and Inf reach
exactly the rows whose neighbourhood holds them, other rows keep their
values); magnitudes that differ by hundreds of decades between x-lines (each
line converted at its own exponent) stay within the parity tolerance; and the
mode y = b - A x of the CG residual."""
import numpy as np
import pytest
import torch

from hpcg_inputs import normal, uniform
from oracle import OracleProblem
from tests.gpu_util import TOL64, dev, host, need_gpu, normwise

pytestmark = pytest.mark.gpu

SHAPES = [(64, 48, 40), (192, 16, 24), (96, 30, 18), (34, 6, 10)]


def _pair(dims, kappa=None):
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    return (HpcgProblem(*dims, levels=1, kappa=None if kappa is None else dev(kappa)),
            OracleProblem(*dims, levels=1, kappa=kappa))


@pytest.mark.parametrize("dims", SHAPES)
def test_unaligned_input_gives_the_same_bits(dims):
    n = int(np.prod(dims))
    g, o = _pair(dims)
    x = normal(n, 301)
    buf = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    buf[1:] = dev(x)
    ya = host(g.spmv(dev(x)))
    yu = host(g.spmv(buf[1:]))  # 8-byte offset: the lines move in 8-byte copies
    np.testing.assert_array_equal(ya, yu)
    assert normwise(ya, o.spmv(x)) <= TOL64


@pytest.mark.parametrize("dims", SHAPES[:2])
def test_nonfinite_and_huge_values(dims):
    n = int(np.prod(dims))
    g, o = _pair(dims)
    nx, ny, nz = dims
    x = normal(n, 302)
    bad = {nx * ny * (nz // 2) + nx * 3 + 5: np.nan, nx * ny * 1 + nx * (ny - 1) + nx - 1: np.inf, 7: 1e300}
    for i, v in bad.items():
        x[i] = v
    y = host(g.spmv(dev(x)))
    with np.errstate(invalid="ignore", over="ignore"):
        yo = o.spmv(x)
    # the same rows are not finite (an infinite x_i makes its own row inf - inf = NaN here, 27 x - S,
    # where the oracle's row sum gives inf), and every NaN of the oracle is a NaN here
    np.testing.assert_array_equal(np.isfinite(y), np.isfinite(yo))
    assert np.all(np.isnan(y[np.isnan(yo)]))
    fin = np.isfinite(yo)
    # rows next to 1e300 carry it; elsewhere the normal parity bound
    near = np.abs(yo) > 1e200
    assert np.all(np.abs(y[fin & near] - yo[fin & near]) <= 1e-12 * np.abs(yo[fin & near]))
    rest = fin & ~near
    assert normwise(y[rest], yo[rest]) <= TOL64


@pytest.mark.parametrize("with_kappa", [False, True])
def test_lines_of_very_different_magnitudes(with_kappa):
    dims = (64, 48, 40)
    nx, ny, nz = dims
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 303) if with_kappa else None
    g, o = _pair(dims, kappa)
    u = np.random.default_rng(304).uniform(-150, 150, size=(nz, ny))
    x = normal(n, 305) * np.repeat((10.0 ** u)[:, :, None], nx, axis=2).reshape(-1)
    y, yo = host(g.spmv(dev(x))), o.spmv(x)
    # each output row against the magnitudes it sums: the largest |x| in its 27-neighbourhood
    m = np.abs(x).reshape(nz, ny, nx)
    pad = np.pad(m, 1)
    nb = np.max([pad[1 + a:1 + a + nz, 1 + b:1 + b + ny, 1 + c:1 + c + nx]
                 for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], axis=0).reshape(-1)
    assert np.all(np.abs(y - yo) <= 1e-13 * 28 * nb)


def test_residual_mode_through_the_solver_start():
    """y = b - A x (the CG start r = b - A x0 and the mixed solver's residual
    replacement) through a solve from a nonzero x0: the first history entry
    divides by ||b - A x0||, so a wrong residual shows in the whole history."""
    dims = (48, 32, 40)
    n = int(np.prod(dims))
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    g = HpcgProblem(*dims, levels=3)
    o = OracleProblem(*dims, levels=3)
    b, x0 = normal(n, 306), normal(n, 307)
    xg, st = g.pcg_solve(dev(b), x0=dev(x0), max_iters=15, tol=0.0)
    xr, hr = o.pcg(b, x0=x0, max_iters=15, tol=0.0)
    h = np.asarray(st.history)
    assert np.max(np.abs(h - hr) / hr) <= 1e-6
    assert normwise(host(xg), xr) <= 1e-10
