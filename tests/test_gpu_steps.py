"""GPU parity of every single step of the hot path against the CPU oracle,
through the C ABI.  Index maps bit-exact; FP64 outputs within 1e-12 normwise."""
import numpy as np
import pytest
import torch

from hpcg_inputs import normal, uniform
from oracle import OracleProblem
from tests.gpu_util import TOL32, TOL64, dev, host, need_gpu, normwise

pytestmark = pytest.mark.gpu

CASES = [((16, 16, 16), 4), ((8, 12, 16), 3), ((2, 2, 2), 1), ((3, 5, 7), 1), ((6, 4, 10), 2), ((64, 32, 48), 4),
         ((34, 18, 66), 2)]


def _pair(dims, levels, kappa=None):
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    g = HpcgProblem(*dims, levels=levels, kappa=None if kappa is None else dev(kappa))
    o = OracleProblem(*dims, levels=levels, kappa=kappa)
    return g, o


@pytest.mark.parametrize("dims,levels", CASES)
def test_setup_maps_bit_exact(dims, levels):
    g, o = _pair(dims, levels)
    for l in range(levels):
        assert g.level_dims(l) == o.dims(l)
        np.testing.assert_array_equal(g.get_colors(l).cpu().numpy(), o.colors(l))
        np.testing.assert_array_equal(g.get_row_nnz(l).cpu().numpy(), o.row_nnz(l))
        if l < levels - 1:
            np.testing.assert_array_equal(g.get_f2c(l).cpu().numpy(), o.f2c(l))
    np.testing.assert_array_equal(host(g.get_rhs()), o.rhs())


@pytest.mark.parametrize("dims,levels", CASES)
@pytest.mark.parametrize("with_kappa", [False, True])
def test_spmv(dims, levels, with_kappa):
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 4) if with_kappa else None
    g, o = _pair(dims, levels, kappa)
    for l in range(levels):
        x = normal(o.n(l), 10 + l)
        y = host(g.spmv(dev(x), level=l))
        assert normwise(y, o.spmv(x, l)) <= TOL64


@pytest.mark.parametrize("dims,levels", CASES)
@pytest.mark.parametrize("with_kappa", [False, True])
def test_colour_steps_and_sweep(dims, levels, with_kappa):
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 4) if with_kappa else None
    g, o = _pair(dims, levels, kappa)
    for l in range(levels):
        r = normal(o.n(l), 20 + l)
        z0 = normal(o.n(l), 30 + l)
        zg = dev(z0)
        zo = z0.copy()
        for k in list(range(8)) + list(range(7, -1, -1)):
            g.rbgs_color(dev(r), zg, k, level=l)
            zo = o.rbgs_color_step(k, r, zo, l)
            assert normwise(host(zg), zo) <= TOL64, (l, k)
        # one whole smoother application (forward then backward colours)
        zs = dev(z0)
        g.rbgs(dev(r), zs, level=l)
        assert normwise(host(zs), o.rbgs(r, z0, l)) <= TOL64


@pytest.mark.parametrize("dims,levels", [c for c in CASES if c[1] > 1])
@pytest.mark.parametrize("with_kappa", [False, True])
def test_restrict_residual_and_prolong(dims, levels, with_kappa):
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 4) if with_kappa else None
    g, o = _pair(dims, levels, kappa)
    for l in range(levels - 1):
        r = normal(o.n(l), 40 + l)
        z = normal(o.n(l), 50 + l)
        rc = host(g.restrict_residual(dev(r), dev(z), level=l))
        ref = o.restrict(r - o.spmv(z, l), l)
        assert normwise(rc, ref) <= TOL64
        zc = normal(o.n(l + 1), 60 + l)
        zg = dev(z)
        g.prolong_add(dev(zc), zg, level=l)
        assert normwise(host(zg), o.prolong_add(zc, z, l)) <= TOL64


@pytest.mark.parametrize("dims,levels", CASES)
@pytest.mark.parametrize("with_kappa", [False, True])
def test_vcycle_fp64(dims, levels, with_kappa):
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 4) if with_kappa else None
    g, o = _pair(dims, levels, kappa)
    r = normal(n, 70)
    z = host(g.mg_vcycle(dev(r)))
    assert normwise(z, o.mg(r)) <= TOL64


def test_dot_and_waxpby():
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    g = HpcgProblem(16, 16, 16, levels=4)
    for n in [0, 1, 255, 256, 257, 4096, 1000003]:
        a, b = normal(n, 1), normal(n, 2)
        d = host(g.dot(dev(a), dev(b)))[0]
        ref = float(np.dot(a, b)) if n else 0.0
        assert abs(d - ref) <= 1e-13 * max(np.abs(a) @ np.abs(b), 1e-300)
        w = host(g.waxpby(1.5, dev(a), -0.25, dev(b)))
        np.testing.assert_allclose(w, 1.5 * a - 0.25 * b, rtol=0, atol=1e-15 * (1 + np.abs(w).max(initial=0.0)))


def test_dot_is_deterministic():
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    g = HpcgProblem(16, 16, 16, levels=4)
    a, b = dev(normal(3000017, 5)), dev(normal(3000017, 6))
    vals = {float(host(g.dot(a, b))[0]) for _ in range(5)}
    assert len(vals) == 1


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vcycle_ignores_stale_buffers(precision):
    """The V-cycle starts every level from z = 0 without clearing memory first:
    lines not yet written count as zero.  A NaN-filled output and a workspace
    left over from a previous call must not leak into the result."""
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    from tests.gpu_util import TOL32
    dims, levels = (32, 24, 16), 3
    n = int(np.prod(dims))
    g = HpcgProblem(*dims, levels=levels, precision=precision)
    o = OracleProblem(*dims, levels=levels)
    tol = TOL64 if precision == "fp64" else TOL32
    z = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    for seed in (1, 2):
        r = normal(n, seed)
        g.mg_vcycle(dev(r), out=z)
        assert normwise(host(z), o.mg(r)) <= tol


def test_autotune_keeps_results():
    """Every launch shape the tuner may pick gives the same bits."""
    import ctypes
    from paper_2304_08232_gb300 import HpcgProblem, _lib
    need_gpu()
    dims = (48, 32, 40)
    n = int(np.prod(dims))
    g = HpcgProblem(*dims, levels=3)
    r = dev(normal(n, 4))
    z1 = host(g.mg_vcycle(r))
    shapes = (ctypes.c_int * 12)()
    lib = _lib.load()
    assert lib.hpcg_autotune(g.h, shapes, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    assert all(v >= 1 for v in shapes)
    z2 = host(g.mg_vcycle(r))
    np.testing.assert_array_equal(z1, z2)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_results_independent_of_launch_shape(precision):
    """Launch shapes only group lines into blocks: SpMV, V-cycle and CG
    results must be bit-identical for any shape (the tuner's choice varies
    from run to run)."""
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    dims = (96, 64, 80)
    n = int(np.prod(dims))
    shapes_a = [[1, 1, 1, 1], [2, 3, 1, 2], [4, 5, 2, 1], [8, 2, 8, 3]]
    shapes_b = [[8, 16, 4, 4], [1, 1, 8, 1], [2, 7, 1, 5], [1, 9, 2, 2]]
    ga = HpcgProblem(*dims, levels=4, precision=precision)
    gb = HpcgProblem(*dims, levels=4, precision=precision)
    ga.set_launch_shapes(shapes_a)
    gb.set_launch_shapes(shapes_b)
    x = dev(normal(n, 21))
    np.testing.assert_array_equal(host(ga.spmv(x)), host(gb.spmv(x)))
    np.testing.assert_array_equal(host(ga.mg_vcycle(x)), host(gb.mg_vcycle(x)))
    b = ga.get_rhs()
    xa, sa = ga.pcg_solve(b, max_iters=12, tol=0.0)
    xb, sb = gb.pcg_solve(b, max_iters=12, tol=0.0)
    np.testing.assert_array_equal(np.asarray(sa.history), np.asarray(sb.history))
    np.testing.assert_array_equal(host(xa), host(xb))


def _random_grids(count, seed):
    """Grids with 1-4 levels, each dimension m 2^(levels-1) with m in 1..9 and at
    least 2 points on the coarsest level (odd coarsest dimensions, dimensions of
    2, x-lines from 2 to 144 points), at most 40,000 rows."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        levels = int(rng.integers(1, 5))
        f = 1 << (levels - 1)
        dims = tuple(int(rng.integers(2 if f == 1 else 1, 10)) * f for _ in range(3))
        if min(d // f for d in dims) < 2 or np.prod(dims) > 40000:
            continue
        out.append((dims, levels))
    return out


@pytest.mark.parametrize("dims,levels", _random_grids(12, 2024))
def test_random_grids_against_oracle(dims, levels):
    """Seeded random grids: setup maps bit-exact; SpMV, one smoother
    application and the V-cycle within 1e-12 of the oracle on every level."""
    g, o = _pair(dims, levels)
    for l in range(levels):
        np.testing.assert_array_equal(host(g.get_colors(l)), o.colors(l))
        n = o.n(l)
        x, r, z0 = normal(n, 81 + l), normal(n, 82 + l), normal(n, 83 + l)
        assert normwise(host(g.spmv(dev(x), l)), o.spmv(x, l)) <= TOL64
        assert normwise(host(g.rbgs(dev(r), dev(z0), l)), o.rbgs(r, z0, l)) <= TOL64
        if l < levels - 1:
            np.testing.assert_array_equal(host(g.get_f2c(l)), o.f2c(l))
    r = normal(o.n(0), 84)
    assert normwise(host(g.mg_vcycle(dev(r))), o.mg(r)) <= TOL64


@pytest.mark.parametrize("dims,levels", _random_grids(6, 2025))
def test_random_grids_mixed_vcycle(dims, levels):
    """The FP32 preconditioner on seeded random grids, within the FP32
    tolerance of the oracle's FP64 V-cycle."""
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    g = HpcgProblem(*dims, levels=levels, precision="mixed")
    o = OracleProblem(*dims, levels=levels)
    r = normal(o.n(0), 85)
    assert normwise(host(g.mg_vcycle(dev(r))), o.mg(r)) <= TOL32
