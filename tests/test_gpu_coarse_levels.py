"""The coarse half of the production V-cycle, stage by stage, against the
oracle (Listing 1; Sec. II-F restriction by injection and its transpose).

With the symmetric colour-ordered smoother and straight injection, the
V-cycle's output hides its coarse levels: the pre-smoother's last colour step
(colour 0) leaves zero residual at the injected points, so the restricted
residual is rounding, and the post-smoother's first step recomputes the
injected points that refinement changed.  These tests therefore observe and
drive every level through hpcg_mg_stage (one stage of Listing 1 with the
V-cycle's own launches, fusions included) and hpcg_get/set_level_vectors:

- the stages run in V-cycle order reproduce hpcg_mg_vcycle bit for bit, so the
  stage calls are the production launches;
- PRE: z_l from a right-hand side set on the level equals the oracle's smoother
  on every level; the fused restriction equals R (r_l - A_l z_l) of the GPU's
  own vectors, point by point, to rounding of the local magnitudes, with
  magnitudes that vary over 80 decades between x-lines so that a coarse value
  taken from the wrong place lands far outside its bound (a shifted oracle
  output must fail the same check);
- REFINE: z_l + R^T z_{l+1} from O(1) vectors set on both levels;
- POST: refinement then post-smoothing against the oracle's composition;
- after a whole V-cycle: each coarse z_l equals the oracle's Listing 1 from
  level l fed the GPU's own r_l, and each r_l is the restricted residual of
  the level above.
Every storage form is covered: block floating point (the default), FP64 z,
mixed precision, the single-launch coarse ends (cluster_tail, persistent) and
the line split over warps (bfp_split).
"""
import numpy as np
import pytest
import torch

from hpcg_inputs import normal, uniform
from oracle import OracleProblem
from tests.gpu_util import TOL32, TOL64, dev, host, need_gpu, normwise

pytestmark = pytest.mark.gpu

# storage form -> HpcgProblem options
MODES = {
    "bfp": {},
    "fp64": {"block_fp": False},
    "mixed": {"precision": "mixed"},
    "cluster": {"cluster_tail": True},
    "persistent": {"persistent": True},
    "persistent_mixed": {"persistent": True, "precision": "mixed"},
    "bfp_split": {"bfp_split": True},  # lines of 65-256 points split over warps (96 x 64 x 80's finest level)
    "planes": {"fuse_planes": 1},  # the runs of one plane parity in one launch (k_gs_planes_bfp)
}
SHAPES = [((16, 16, 16), 4), ((64, 32, 48), 4), ((96, 64, 80), 4)]
EPS64 = np.finfo(np.float64).eps
EPS32 = float(np.finfo(np.float32).eps)


def _tol(mode):
    return TOL32 if "mixed" in mode else TOL64


def _eps(mode):
    return EPS32 if "mixed" in mode else EPS64


def _problem(dims, levels, mode, kappa=None):
    from paper_2304_08232_gb300 import HpcgProblem
    need_gpu()
    return HpcgProblem(*dims, levels=levels, kappa=None if kappa is None else dev(kappa), **MODES[mode])


def _get(g, l, r=False, z=True):
    rt, zt = g.get_level_vectors(l, r=r, z=z)
    return (host(rt) if rt is not None else None), (host(zt) if zt is not None else None)


def _level_z(g, l, z0, mode):
    """z_l as the stage left it (level 0 with FP64 storage: the caller's z0)."""
    if l == 0 and mode in ("fp64", "persistent"):
        return host(z0)
    return _get(g, l)[1]


def _set_r(g, l, r):
    g.set_level_vectors(l, r=dev(r))
    return _get(g, l, r=True, z=False)[0]


def _set_z(g, l, z, z0, mode):
    if l == 0 and mode in ("fp64", "persistent"):
        z0.copy_(dev(z))
        return host(z0)
    g.set_level_vectors(l, z=dev(z))
    return _get(g, l)[1]


def _line_spread(dims, seed, decades=40.0):
    """A factor 10^u per x-line, u ~ U[-decades, decades] (seeded)."""
    nx, ny, nz = dims
    u = np.random.default_rng(seed).uniform(-decades, decades, size=(nz, ny))
    return np.repeat((10.0 ** u)[:, :, None], nx, axis=2).reshape(-1)


def _restrict_bound(dims, r, z, c_eps):
    """Per coarse point: c_eps times the largest |r| or |z| on the 3 x 3 fine
    x-lines around the fine line of its injected point (the magnitudes that the
    restricted residual's rounding scales with)."""
    nx, ny, nz = dims
    m = np.maximum(np.abs(r), np.abs(z)).reshape(nz, ny, nx).max(axis=2)
    pad = np.pad(m, 1)
    nb = np.max([pad[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny] for dz in (-1, 0, 1) for dy in (-1, 0, 1)], axis=0)
    cb = nb[0::2, 0::2]  # fine line (2 yc, 2 zc) of coarse line (yc, zc)
    return c_eps * np.repeat(cb[:, :, None], nx // 2, axis=2).reshape(-1)


def _restriction_ok(o, l, dims, r, z, rc_gpu, c_eps, shift=0, drop_az=False):
    """rc_gpu against R (r - A z) of the same vectors (oracle), point by point.
    Planted oracle mistakes: shift != 0 moves the oracle's output by that many
    coarse x-lines; drop_az restricts r alone."""
    ref = o.restrict(r - (0.0 if drop_az else o.spmv(z, l)), l)
    if shift:
        nc = dims[0] // 2
        ref = np.roll(ref, shift * nc)
    bound = _restrict_bound(dims, r, z, c_eps)
    return bool(np.all(np.abs(rc_gpu - ref) <= bound)), ref


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("dims,levels", SHAPES[:2])
def test_stages_in_vcycle_order_are_the_vcycle(mode, dims, levels):
    n = int(np.prod(dims))
    g = _problem(dims, levels, mode)
    r = dev(normal(n, 61))
    z_ref = host(g.mg_vcycle(r))
    z = torch.full_like(r, np.nan)
    for l in range(levels):
        g.mg_stage(l, "pre", r, z)
    for l in range(levels - 2, -1, -1):
        g.mg_stage(l, "post", r, z)
    np.testing.assert_array_equal(host(z), z_ref)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("dims,levels", SHAPES)
@pytest.mark.parametrize("with_kappa", [False, True])
def test_pre_stage_smoother_and_fused_restriction(mode, dims, levels, with_kappa):
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 62) if with_kappa else None
    g = _problem(dims, levels, mode, kappa)
    o = OracleProblem(*dims, levels=levels, kappa=kappa)
    tol, eps = _tol(mode), _eps(mode)
    r0 = dev(normal(n, 63))
    z0 = torch.zeros_like(r0)
    for l in range(levels):
        dl = o.dims(l)
        nl = int(np.prod(dl))
        if l == 0:
            rl = host(r0)
        else:
            rl = _set_r(g, l, normal(nl, 64 + l))
        g.mg_stage(l, "pre", r0, z0)
        zl = _level_z(g, l, z0, mode)
        assert normwise(zl, o.rbgs(rl, np.zeros(nl), l)) <= tol, (mode, l)
        if l < levels - 1:
            rc = _get(g, l + 1, r=True, z=False)[0]
            ok, ref = _restriction_ok(o, l, dl, rl, zl, rc, 256 * eps)
            assert ok, (mode, l, np.abs(rc - ref).max())


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("dims,levels", SHAPES[1:])
def test_fused_restriction_lands_on_its_coarse_points(mode, dims, levels):
    """Right-hand sides whose magnitudes differ by up to 80 decades between
    x-lines (30 in FP32 range for mixed precision): each restricted value must
    be rounding of its own neighbourhood's magnitude.  The same check on a
    planted oracle mistake must fail: the output shifted by one coarse line
    (FP64 forms, where the oracle's rounding and the kernels' are alike), or
    r restricted without A z (every form; in FP32 the kernels' rounding is
    2^29 times the oracle's, so a shifted FP64 output of rounding size would
    still fit the FP32 bound)."""
    n = int(np.prod(dims))
    g = _problem(dims, levels, mode)
    o = OracleProblem(*dims, levels=levels)
    eps = _eps(mode)
    dec = 15.0 if "mixed" in mode else 40.0
    r0 = dev(normal(n, 71) * _line_spread(dims, 72, dec))
    z0 = torch.zeros_like(r0)
    for l in range(levels - 1):
        dl = o.dims(l)
        nl = int(np.prod(dl))
        rl = host(r0) if l == 0 else _set_r(g, l, normal(nl, 73 + l) * _line_spread(dl, 74 + l, dec))
        g.mg_stage(l, "pre", r0, z0)
        zl = _level_z(g, l, z0, mode)
        rc = _get(g, l + 1, r=True, z=False)[0]
        ok, ref = _restriction_ok(o, l, dl, rl, zl, rc, 256 * eps)
        assert ok, (mode, l)
        if "mixed" not in mode:
            assert not _restriction_ok(o, l, dl, rl, zl, rc, 256 * eps, shift=1)[0], (mode, l)
        assert not _restriction_ok(o, l, dl, rl, zl, rc, 256 * eps, drop_az=True)[0], (mode, l)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("dims,levels", SHAPES)
def test_refine_stage_adds_the_coarse_correction(mode, dims, levels):
    n = int(np.prod(dims))
    g = _problem(dims, levels, mode)
    o = OracleProblem(*dims, levels=levels)
    r0 = dev(normal(n, 81))
    z0 = torch.zeros_like(r0)
    for l in range(levels - 2, -1, -1):
        nl, nc = o.n(l), o.n(l + 1)
        zc = _set_z(g, l + 1, normal(nc, 82 + l), z0, mode)
        zf = _set_z(g, l, normal(nl, 90 + l), z0, mode)
        g.mg_stage(l, "refine", r0, z0)
        out = _level_z(g, l, z0, mode)
        ref = o.prolong_add(zc, zf, l)
        assert normwise(out, ref) <= _tol(mode), (mode, l)
        # points that are not injected keep their values (to the rounding of the common exponent)
        inj = np.zeros(nl, dtype=bool)
        inj[o.f2c(l)] = True
        assert np.max(np.abs(out[~inj] - zf[~inj])) <= 4 * _eps(mode) * np.abs(zf).max()


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("dims,levels", SHAPES)
@pytest.mark.parametrize("with_kappa", [False, True])
def test_post_stage_is_refinement_then_smoother(mode, dims, levels, with_kappa):
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 100) if with_kappa else None
    g = _problem(dims, levels, mode, kappa)
    o = OracleProblem(*dims, levels=levels, kappa=kappa)
    r0 = dev(normal(n, 101))
    z0 = torch.zeros_like(r0)
    for l in range(levels - 2, -1, -1):
        nl, nc = o.n(l), o.n(l + 1)
        rl = host(r0) if l == 0 else _set_r(g, l, normal(nl, 102 + l))
        zc = _set_z(g, l + 1, normal(nc, 110 + l), z0, mode)
        zf = _set_z(g, l, normal(nl, 120 + l), z0, mode)
        g.mg_stage(l, "post", r0, z0)
        out = _level_z(g, l, z0, mode)
        ref = o.rbgs(rl, o.prolong_add(zc, zf, l), l)
        assert normwise(out, ref) <= _tol(mode), (mode, l)
        if l == 0 and mode not in ("fp64", "persistent"):
            assert normwise(host(z0), ref) <= _tol(mode)  # the FP64 result the V-cycle returns


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("dims,levels", SHAPES)
@pytest.mark.parametrize("with_kappa", [False, True])
def test_coarse_levels_after_a_whole_vcycle(mode, dims, levels, with_kappa):
    """After hpcg_mg_vcycle: z_l (l >= 1) is Listing 1 from level l on the
    GPU's own r_l, and r_l is the restricted residual of the pre-smoothed
    level above (the oracle's smoother on the GPU's r_{l-1})."""
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 130) if with_kappa else None
    g = _problem(dims, levels, mode, kappa)
    o = OracleProblem(*dims, levels=levels, kappa=kappa)
    r = normal(n, 131)
    g.mg_vcycle(dev(r))
    torch.cuda.synchronize()
    eps = _eps(mode)
    r_prev = r
    for l in range(1, levels):
        rl, zl = _get(g, l, r=True, z=True)
        assert normwise(zl, o.mg(rl, l)) <= _tol(mode), (mode, l)
        dp = o.dims(l - 1)
        zp = o.rbgs(r_prev, np.zeros(o.n(l - 1)), l - 1)
        ok, ref = _restriction_ok(o, l - 1, dp, r_prev, zp, rl, 1024 * eps)
        assert ok, (mode, l, np.abs(rl - ref).max())
        r_prev = rl


@pytest.mark.slow
@pytest.mark.parametrize("with_kappa", [False, True])
def test_coarse_levels_at_192cubed(with_kappa):
    """The bench's grid: levels 1-3 of 192^3 (96^3, 48^3, 24^3) checked with an
    oracle hierarchy built on 96^3 (the same coarse operators: each level
    regenerates the stencil, kappa injected from the level above), level 0's
    fused restriction on every injected row with the oracle's row generator."""
    from oracle import spmv_rows
    dims, levels = (192, 192, 192), 4
    n = int(np.prod(dims))
    kappa = uniform(n, 0.0, 1.0, 140) if with_kappa else None
    g = _problem(dims, levels, "bfp", kappa)
    r0 = dev(normal(n, 141))
    z0 = torch.zeros_like(r0)
    g.mg_stage(0, "pre", r0, z0)
    z_pre = _get(g, 0)[1]
    r1 = _get(g, 1, r=True, z=False)[0]
    # level-0 restriction: r - A z at every injected row (2 xc, 2 yc, 2 zc)
    h = np.arange(96)
    inj = (2 * h[None, None, :] + 192 * (2 * h[None, :, None] + 192 * 2 * h[:, None, None])).reshape(-1)
    rh = host(r0)
    ref = rh[inj] - spmv_rows(*dims, inj, z_pre, kappa)
    bound = _restrict_bound(dims, rh, z_pre, 256 * EPS64)
    assert np.all(np.abs(r1 - ref) <= bound)
    # whole V-cycle, then levels 1..3 against the 96^3 oracle hierarchy
    g.mg_vcycle(r0)
    torch.cuda.synchronize()
    kc = kappa.reshape(192, 192, 192)[0::2, 0::2, 0::2].reshape(-1) if with_kappa else None
    o = OracleProblem(96, 96, 96, levels=3, kappa=kc)
    r_prev = None
    for l in range(1, levels):
        rl, zl = _get(g, l, r=True, z=True)
        assert normwise(zl, o.mg(rl, l - 1)) <= TOL64, l
        if r_prev is not None:
            zp = o.rbgs(r_prev, np.zeros(o.n(l - 2)), l - 2)
            ok, _ = _restriction_ok(o, l - 2, o.dims(l - 2), r_prev, zp, rl, 1024 * EPS64)
            assert ok, l
        r_prev = rl


def test_stage_argument_errors():
    from paper_2304_08232_gb300._lib import HpcgError
    g = _problem((16, 16, 16), 4, "bfp")
    r = dev(normal(4096, 150))
    z = torch.zeros_like(r)
    with pytest.raises(HpcgError):
        g.mg_stage(3, "post", r, z)  # the coarsest level has no coarser one
    assert g.lib.hpcg_mg_stage(g.h, 0, 0, None, None, None) == 1  # level 0 needs r0 and z0 (INVALID_ARG)
    assert g.lib.hpcg_mg_stage(g.h, 1, 3, None, None, None) == 1  # no such stage
    with pytest.raises(HpcgError):
        g.get_level_vectors(0, r=True)  # r_0 is the caller's
    gf = _problem((16, 16, 16), 4, "fp64")
    with pytest.raises(HpcgError):
        gf.get_level_vectors(0, r=False, z=True)  # FP64 storage keeps z_0 in the caller's buffer
