"""Thin torch-facing wrappers with the names of the C ABI (include/hpcg.h)."""
import ctypes

import torch

from . import _lib
from ._lib import check, hpcg_options, hpcg_stats

_f64 = torch.float64


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t, n, dtype=_f64, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError("%s must be contiguous %s with %d elements" % (name, dtype, n))
    return t


def launch_count():
    return _lib.load().hpcg_launch_count()


class _Stats:
    """Host-side statistics of one solve (iterations, residual history)."""

    def __init__(self, st, hist):
        self.iters = st.iters
        self.restarts = st.restarts
        self.converged = bool(st.converged)
        self.status = st.status
        self.rel_res = st.rel_res
        self.history = hist[: st.iters].tolist() if hist is not None else []

    def __repr__(self):
        return "Stats(iters=%d, rel_res=%.3e, converged=%s, restarts=%d)" % (
            self.iters, self.rel_res, self.converged, self.restarts)


def _new_stats(cap):
    import numpy as np
    hist = np.zeros(max(cap, 1), dtype=np.float64)
    st = hpcg_stats()
    st.history = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st.history_cap = len(hist)
    return st, hist


class HpcgProblem:
    """One grid hierarchy (hpcg_setup_ex) with a torch-allocated workspace."""

    def __init__(self, nx, ny, nz, levels=4, precision="fp64", kappa=None, pre_sweeps=1, post_sweeps=1,
                 symmetric=True, max_rhs=0, check_every=1, persistent=False, fixed_point=True, pdl=True, block_fp=True,
                 cluster_tail=False, restart_every=0, bfp_split=False, fuse_planes=0, device=None,
                 lib=None):
        self.lib = lib if lib is not None else _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("HpcgProblem needs a CUDA device")
        self.device = torch.device(device or "cuda")
        opt = hpcg_options()
        check(self.lib.hpcg_options_default(ctypes.byref(opt), nx, ny, nz), "hpcg_options_default")
        opt.levels = levels
        opt.precision = {"fp64": _lib.FP64, "mixed": _lib.MIXED}[precision]
        opt.pre_sweeps, opt.post_sweeps = pre_sweeps, post_sweeps
        opt.symmetric = 1 if symmetric else 0
        opt.max_rhs = max_rhs
        opt.check_every = check_every
        opt.persistent = 1 if persistent else 0
        opt.fixed_point = 1 if fixed_point else 0
        opt.pdl = 1 if pdl else 0
        opt.block_fp = 1 if block_fp else 0
        opt.cluster_tail = 1 if cluster_tail else 0
        opt.restart_every = int(restart_every)
        opt.bfp_split = 1 if bfp_split else 0
        opt.fuse_planes = int(fuse_planes)
        self.dims = (nx, ny, nz)
        self.levels = levels
        self.precision = precision
        self.n = nx * ny * nz
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.hpcg_setup_ex(ctypes.byref(opt), None, ctypes.byref(h)), "hpcg_setup_ex")
            self.h = h
            nbytes = ctypes.c_size_t()
            check(self.lib.hpcg_workspace_bytes(self.h, ctypes.byref(nbytes)), "hpcg_workspace_bytes")
            self.workspace = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
            base = self.workspace.data_ptr()
            aligned = (base + 255) & ~255
            check(self.lib.hpcg_bind_workspace(self.h, ctypes.c_void_p(aligned), nbytes.value), "hpcg_bind_workspace")
            if kappa is not None:
                self.set_kappa(kappa)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                self.lib.hpcg_destroy(h)
            except Exception:
                pass
            self.h = None

    # -- geometry / maps --------------------------------------------------------
    def level_dims(self, level):
        d = (ctypes.c_int * 3)()
        check(self.lib.hpcg_level_dims(self.h, level, d), "hpcg_level_dims")
        return tuple(d)

    def level_n(self, level):
        a, b, c = self.level_dims(level)
        return a * b * c

    def autotune(self):
        """Re-times the line-kernel launch shapes; returns them per level."""
        buf = (ctypes.c_int * (4 * self.levels))()
        check(self.lib.hpcg_autotune(self.h, buf, _stream()), "hpcg_autotune")
        return [list(buf[4 * l:4 * l + 4]) for l in range(self.levels)]

    def set_launch_shapes(self, shapes):
        flat = [int(v) for lv in shapes for v in lv]
        buf = (ctypes.c_int * len(flat))(*flat)
        check(self.lib.hpcg_set_launch_shapes(self.h, buf), "hpcg_set_launch_shapes")

    def profile_iteration(self, b, x0=None):
        """Per-level / per-kernel-class milliseconds of one CG iteration
        (hpcg_profile_iteration); x0 is left untouched (a copy is iterated)."""
        _need(b, self.n, name="b")
        x = x0.clone() if x0 is not None else torch.zeros_like(b)
        L = self.levels
        buf = (ctypes.c_double * (3 * L + 7))()
        check(self.lib.hpcg_profile_iteration(self.h, _ptr(b), _ptr(x), buf, 3 * L + 7, _stream()),
              "hpcg_profile_iteration")
        v = list(buf)
        return {"smoother_ms": v[0:L], "restriction_ms": v[L:2 * L], "refinement_ms": v[2 * L:3 * L],
                "persistent_coarse_ms": v[3 * L], "spmv_ms": v[3 * L + 1], "dot_ms": v[3 * L + 2],
                "update_ms": v[3 * L + 3], "finalize_ms": v[3 * L + 4], "convert_ms": v[3 * L + 5],
                "total_ms": v[3 * L + 6]}

    def set_kappa(self, kappa):
        if kappa is not None:
            kappa = _need(kappa, self.n, name="kappa")
        check(self.lib.hpcg_set_kappa(self.h, _ptr(kappa), _stream()), "hpcg_set_kappa")
        self._kappa_ref = kappa

    def get_colors(self, level=0):
        out = torch.empty(self.level_n(level), dtype=torch.int32, device=self.device)
        check(self.lib.hpcg_get_colors(self.h, level, _ptr(out), _stream()), "hpcg_get_colors")
        return out

    def get_f2c(self, level=0):
        out = torch.empty(self.level_n(level + 1), dtype=torch.int32, device=self.device)
        check(self.lib.hpcg_get_f2c(self.h, level, _ptr(out), _stream()), "hpcg_get_f2c")
        return out

    def get_row_nnz(self, level=0):
        out = torch.empty(self.level_n(level), dtype=torch.int32, device=self.device)
        check(self.lib.hpcg_get_row_nnz(self.h, level, _ptr(out), _stream()), "hpcg_get_row_nnz")
        return out

    def get_rhs(self):
        out = torch.empty(self.n, dtype=_f64, device=self.device)
        check(self.lib.hpcg_get_rhs(self.h, _ptr(out), _stream()), "hpcg_get_rhs")
        return out

    # -- single steps -----------------------------------------------------------------
    def spmv(self, x, level=0, out=None):
        n = self.level_n(level)
        _need(x, n, name="x")
        out = torch.empty_like(x) if out is None else _need(out, n, name="out")
        check(self.lib.hpcg_spmv(self.h, level, _ptr(x), _ptr(out), _stream()), "hpcg_spmv")
        return out

    def rbgs_color(self, r, z, color, level=0):
        n = self.level_n(level)
        _need(r, n, name="r"), _need(z, n, name="z")
        check(self.lib.hpcg_rbgs_color(self.h, level, color, _ptr(r), _ptr(z), _stream()), "hpcg_rbgs_color")
        return z

    def rbgs(self, r, z, level=0):
        n = self.level_n(level)
        _need(r, n, name="r"), _need(z, n, name="z")
        check(self.lib.hpcg_rbgs(self.h, level, _ptr(r), _ptr(z), _stream()), "hpcg_rbgs")
        return z

    def restrict_residual(self, r, z, level=0, out=None):
        n = self.level_n(level)
        _need(r, n, name="r"), _need(z, n, name="z")
        nc = self.level_n(level + 1)
        out = torch.empty(nc, dtype=_f64, device=self.device) if out is None else _need(out, nc, name="out")
        check(self.lib.hpcg_restrict_residual(self.h, level, _ptr(r), _ptr(z), _ptr(out), _stream()),
              "hpcg_restrict_residual")
        return out

    def prolong_add(self, zc, z, level=0):
        _need(zc, self.level_n(level + 1), name="zc"), _need(z, self.level_n(level), name="z")
        check(self.lib.hpcg_prolong_add(self.h, level, _ptr(zc), _ptr(z), _stream()), "hpcg_prolong_add")
        return z

    def mg_vcycle(self, r, out=None):
        _need(r, self.n, name="r")
        out = torch.empty_like(r) if out is None else _need(out, self.n, name="out")
        check(self.lib.hpcg_mg_vcycle(self.h, _ptr(r), _ptr(out), _stream()), "hpcg_mg_vcycle")
        return out

    # -- the V-cycle stage by stage (hpcg_mg_stage) and its level vectors ---------------
    def mg_stage(self, level, stage, r0=None, z0=None):
        """One stage ("pre", "refine" or "post") of Listing 1 on `level`, on the
        handle's level vectors; level 0 takes r0 and z0 (FP64 [n_0])."""
        code = {"pre": _lib.STAGE_PRE, "refine": _lib.STAGE_REFINE, "post": _lib.STAGE_POST}[stage]
        if level == 0:
            _need(r0, self.n, name="r0"), _need(z0, self.n, name="z0")
        check(self.lib.hpcg_mg_stage(self.h, level, code, _ptr(r0) if level == 0 else None,
                                     _ptr(z0) if level == 0 else None, _stream()), "hpcg_mg_stage")
        return z0

    def get_level_vectors(self, level, r=True, z=True):
        """(r_l, z_l) as FP64 tensors (None where not asked for)."""
        n = self.level_n(level)
        rt = torch.empty(n, dtype=_f64, device=self.device) if r else None
        zt = torch.empty(n, dtype=_f64, device=self.device) if z else None
        check(self.lib.hpcg_get_level_vectors(self.h, level, _ptr(rt), _ptr(zt), _stream()), "hpcg_get_level_vectors")
        return rt, zt

    def set_level_vectors(self, level, r=None, z=None):
        n = self.level_n(level)
        if r is not None:
            _need(r, n, name="r")
        if z is not None:
            _need(z, n, name="z")
        check(self.lib.hpcg_set_level_vectors(self.h, level, _ptr(r), _ptr(z), _stream()), "hpcg_set_level_vectors")

    def dot(self, a, b):
        out = torch.empty(1, dtype=_f64, device=self.device)
        check(self.lib.hpcg_dot(self.h, a.numel(), _ptr(a), _ptr(b), _ptr(out), _stream()), "hpcg_dot")
        return out

    def waxpby(self, alpha, x, beta, y, out=None):
        out = torch.empty_like(x) if out is None else out
        check(self.lib.hpcg_waxpby(self.h, x.numel(), alpha, _ptr(x), beta, _ptr(y), _ptr(out), _stream()),
              "hpcg_waxpby")
        return out

    # -- solves --------------------------------------------------------------------------
    def pcg_solve(self, b, x0=None, max_iters=50, tol=0.0, out=None):
        """Returns (x, stats).  tol <= 0 runs exactly max_iters iterations."""
        _need(b, self.n, name="b")
        x = out if out is not None else (x0.clone() if x0 is not None else torch.zeros_like(b))
        if out is not None and x0 is not None:
            x.copy_(x0)
        st, hist = _new_stats(max_iters)
        rc = self.lib.hpcg_pcg_solve(self.h, _ptr(b), _ptr(x), max_iters, tol, ctypes.byref(st), _stream())
        check(rc, "hpcg_pcg_solve", allow=(_lib.HPCG_ERR_NOT_CONVERGED,))
        return x, _Stats(st, hist)

    def pcg_backward(self, x, grad_x, max_iters=200, tol=1e-12, want_kappa=True):
        _need(x, self.n, name="x"), _need(grad_x, self.n, name="grad_x")
        gb = torch.empty_like(x)
        gk = torch.empty_like(x) if want_kappa else None
        st, hist = _new_stats(max_iters)
        rc = self.lib.hpcg_pcg_backward(self.h, _ptr(x), _ptr(grad_x), _ptr(gb), _ptr(gk), max_iters, tol,
                                        ctypes.byref(st), _stream())
        check(rc, "hpcg_pcg_backward", allow=(_lib.HPCG_ERR_NOT_CONVERGED,))
        return gb, gk, _Stats(st, hist)

    def pcg_solve_multi(self, B, X0=None, max_iters=50, tol=0.0):
        nrhs = B.shape[0]
        _need(B, nrhs * self.n, name="B")
        X = X0.clone() if X0 is not None else torch.zeros_like(B)
        sts = (hpcg_stats * nrhs)()
        hists = []
        for k in range(nrhs):
            st, hist = _new_stats(max_iters)
            sts[k] = st
            hists.append(hist)
        rc = self.lib.hpcg_pcg_solve_multi(self.h, nrhs, _ptr(B), _ptr(X), max_iters, tol, sts, _stream())
        check(rc, "hpcg_pcg_solve_multi", allow=(_lib.HPCG_ERR_NOT_CONVERGED,))
        return X, [_Stats(sts[k], hists[k]) for k in range(nrhs)]


class HpcgEll:
    """The operator stored as a sliced-ELL matrix with rows grouped by colour
    (P^T A P, hpcg_ell_setup); colour_sorted=False keeps the natural order.
    Level calls take vectors in the stored order (to_stored / to_natural)."""

    def __init__(self, nx, ny, nz, levels=4, colour_sorted=True, exact=False, bf16_values=False, device=None):
        self.lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("HpcgEll needs a CUDA device")
        self.device = torch.device(device or "cuda")
        self.dims, self.levels = (nx, ny, nz), levels
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.hpcg_ell_setup(nx, ny, nz, levels, 1 if colour_sorted else 0, 1 if exact else 0, 1 if bf16_values else 0,
                                          ctypes.byref(h)), "hpcg_ell_setup")
        self.h = h
        self.n = nx * ny * nz

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                self.lib.hpcg_ell_destroy(h)
            except Exception:
                pass
            self.h = None

    def nbytes(self):
        v = ctypes.c_size_t()
        check(self.lib.hpcg_ell_bytes(self.h, ctypes.byref(v)), "hpcg_ell_bytes")
        return v.value

    def level_info(self, level=0):
        """(rows, slices, cstart[0..8])"""
        buf = (ctypes.c_long * 11)()
        check(self.lib.hpcg_ell_level_info(self.h, level, buf), "hpcg_ell_level_info")
        return buf[0], buf[1], list(buf[2:11])

    def permutation(self, level=0):
        n = self.level_info(level)[0]
        out = torch.empty(n, dtype=torch.int32, device=self.device)
        check(self.lib.hpcg_ell_permutation(self.h, level, _ptr(out), _stream()), "hpcg_ell_permutation")
        return out

    def matrix(self, level=0):
        """(col, val) of the slices, slot s of stored row p at ((p//32)*27 + s)*32 + p%32."""
        slices = self.level_info(level)[1]
        col = torch.empty(slices * 27 * 32, dtype=torch.int32, device=self.device)
        val = torch.empty(slices * 27 * 32, dtype=_f64, device=self.device)
        check(self.lib.hpcg_ell_matrix(self.h, level, _ptr(col), _ptr(val), _stream()), "hpcg_ell_matrix")
        return col, val

    def _n(self, level):
        return self.level_info(level)[0]

    def to_stored(self, v, level=0):
        n = self._n(level)
        _need(v, n, name="v")
        out = torch.empty_like(v)
        check(self.lib.hpcg_ell_permute(self.h, level, 1, _ptr(v), _ptr(out), _stream()), "hpcg_ell_permute")
        return out

    def to_natural(self, v, level=0):
        n = self._n(level)
        _need(v, n, name="v")
        out = torch.empty_like(v)
        check(self.lib.hpcg_ell_permute(self.h, level, 0, _ptr(v), _ptr(out), _stream()), "hpcg_ell_permute")
        return out

    def spmv(self, x, level=0, out=None):
        n = self._n(level)
        _need(x, n, name="x")
        out = torch.empty_like(x) if out is None else _need(out, n, name="out")
        check(self.lib.hpcg_ell_spmv(self.h, level, _ptr(x), _ptr(out), _stream()), "hpcg_ell_spmv")
        return out

    def rbgs_color(self, r, z, color, level=0):
        n = self._n(level)
        _need(r, n, name="r"), _need(z, n, name="z")
        check(self.lib.hpcg_ell_rbgs_color(self.h, level, color, _ptr(r), _ptr(z), _stream()), "hpcg_ell_rbgs_color")
        return z

    def rbgs(self, r, z, level=0):
        n = self._n(level)
        _need(r, n, name="r"), _need(z, n, name="z")
        check(self.lib.hpcg_ell_rbgs(self.h, level, _ptr(r), _ptr(z), _stream()), "hpcg_ell_rbgs")
        return z

    def mg_vcycle(self, r, out=None):
        _need(r, self.n, name="r")
        out = torch.empty_like(r) if out is None else _need(out, self.n, name="out")
        check(self.lib.hpcg_ell_mg_vcycle(self.h, _ptr(r), _ptr(out), _stream()), "hpcg_ell_mg_vcycle")
        return out

    def pcg_solve(self, b, x0=None, max_iters=50, tol=0.0, out=None):
        """b, x in natural order; returns (x, stats)."""
        _need(b, self.n, name="b")
        x = out if out is not None else (x0.clone() if x0 is not None else torch.zeros_like(b))
        if out is not None:
            if x0 is not None:
                x.copy_(x0)
            else:
                x.zero_()
        st, hist = _new_stats(max_iters)
        rc = self.lib.hpcg_ell_pcg_solve(self.h, _ptr(b), _ptr(x), max_iters, tol, ctypes.byref(st), _stream())
        check(rc, "hpcg_ell_pcg_solve", allow=(_lib.HPCG_ERR_NOT_CONVERGED,))
        return x, _Stats(st, hist)


class HpcgSplit:
    """One grid as two z-slabs with their own rows and halos and colour-aware
    halo exchange (hpcg_split_setup), run on one GPU; natural-order vectors."""

    def __init__(self, nx, ny, nz, levels=4, exact=False, device=None):
        self.lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("HpcgSplit needs a CUDA device")
        self.device = torch.device(device or "cuda")
        self.dims, self.levels = (nx, ny, nz), levels
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.hpcg_split_setup(nx, ny, nz, levels, 1 if exact else 0, ctypes.byref(h)), "hpcg_split_setup")
        self.h = h
        self.n = nx * ny * nz

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                self.lib.hpcg_split_destroy(h)
            except Exception:
                pass
            self.h = None

    def info(self, level, domain):
        """dict: z range, own rows, halo rows, colour starts of own and halo rows"""
        b = (ctypes.c_long * 22)()
        check(self.lib.hpcg_split_info(self.h, level, domain, b), "hpcg_split_info")
        return {"z": (b[0], b[1]), "own": b[2], "halo": b[3], "cstart": list(b[4:13]), "hstart": list(b[13:22])}

    def exchange_count(self):
        v, s_ = ctypes.c_long(), ctypes.c_long()
        check(self.lib.hpcg_split_exchange_count(self.h, ctypes.byref(v), ctypes.byref(s_)), "hpcg_split_exchange_count")
        return v.value, s_.value

    def _n(self, level):
        return (self.dims[0] >> level) * (self.dims[1] >> level) * (self.dims[2] >> level)

    def spmv(self, x, level=0, out=None):
        n = self._n(level)
        _need(x, n, name="x")
        out = torch.empty_like(x) if out is None else _need(out, n, name="out")
        check(self.lib.hpcg_split_spmv(self.h, level, _ptr(x), _ptr(out), _stream()), "hpcg_split_spmv")
        return out

    def rbgs(self, r, z, level=0):
        n = self._n(level)
        _need(r, n, name="r"), _need(z, n, name="z")
        check(self.lib.hpcg_split_rbgs(self.h, level, _ptr(r), _ptr(z), _stream()), "hpcg_split_rbgs")
        return z

    def mg_vcycle(self, r, out=None):
        _need(r, self.n, name="r")
        out = torch.empty_like(r) if out is None else _need(out, self.n, name="out")
        check(self.lib.hpcg_split_mg_vcycle(self.h, _ptr(r), _ptr(out), _stream()), "hpcg_split_mg_vcycle")
        return out

    def pcg_solve(self, b, x0=None, max_iters=50, tol=0.0, out=None):
        _need(b, self.n, name="b")
        x = out if out is not None else (x0.clone() if x0 is not None else torch.zeros_like(b))
        if out is not None:
            if x0 is not None:
                x.copy_(x0)
            else:
                x.zero_()
        st, hist = _new_stats(max_iters)
        rc = self.lib.hpcg_split_pcg_solve(self.h, _ptr(b), _ptr(x), max_iters, tol, ctypes.byref(st), _stream())
        check(rc, "hpcg_split_pcg_solve", allow=(_lib.HPCG_ERR_NOT_CONVERGED,))
        return x, _Stats(st, hist)


class HpcgBatch:
    """A batch of independent grids (hpcg_setup_batch), vectors concatenated."""

    def __init__(self, dims, levels=4, precision="fp64", device=None, lib=None):
        self.lib = lib if lib is not None else _lib.load()
        self.device = torch.device(device or "cuda")
        flat = [int(v) for d in dims for v in d]
        self.count = len(dims)
        arr = (ctypes.c_int * len(flat))(*flat)
        h = ctypes.c_void_p()
        prec = {"fp64": _lib.FP64, "mixed": _lib.MIXED}[precision]
        with torch.cuda.device(self.device):
            check(self.lib.hpcg_setup_batch(self.count, arr, levels, prec, ctypes.byref(h)), "hpcg_setup_batch")
            self.h = h
            offs = (ctypes.c_long * (self.count + 1))()
            check(self.lib.hpcg_batch_offsets(self.h, offs), "hpcg_batch_offsets")
            self.offsets = list(offs)
            self.n = self.offsets[-1]
            nbytes = ctypes.c_size_t()
            check(self.lib.hpcg_workspace_bytes(self.h, ctypes.byref(nbytes)), "hpcg_workspace_bytes")
            self.workspace = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
            aligned = (self.workspace.data_ptr() + 255) & ~255
            check(self.lib.hpcg_bind_workspace(self.h, ctypes.c_void_p(aligned), nbytes.value), "hpcg_bind_workspace")

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                self.lib.hpcg_destroy(h)
            except Exception:
                pass
            self.h = None

    def pcg_solve(self, b, x0=None, max_iters=200, tol=1e-8):
        _need(b, self.n, name="b")
        x = x0.clone() if x0 is not None else torch.zeros_like(b)
        sts = (hpcg_stats * self.count)()
        hists = []
        for k in range(self.count):
            st, hist = _new_stats(max_iters)
            sts[k] = st
            hists.append(hist)
        rc = self.lib.hpcg_pcg_solve_batch(self.h, _ptr(b), _ptr(x), max_iters, tol, sts, _stream())
        check(rc, "hpcg_pcg_solve_batch", allow=(_lib.HPCG_ERR_NOT_CONVERGED,))
        return x, [_Stats(sts[k], hists[k]) for k in range(self.count)]


class HpcgSolve(torch.autograd.Function):
    """x = A(kappa)^{-1} b with a hand-written backward: the adjoint MG-PCG
    solve lambda = A^{-1} grad_x (A is symmetric), grad_b = lambda and
    grad_kappa = -lambda * x (hpcg_pcg_backward)."""

    @staticmethod
    def forward(ctx, b, kappa, problem, max_iters, tol):
        kd = kappa.detach().contiguous()
        problem.set_kappa(kd)
        x, st = problem.pcg_solve(b.detach().contiguous(), max_iters=max_iters, tol=tol)
        ctx.problem, ctx.max_iters, ctx.tol = problem, max_iters, tol
        # kappa is saved too (autograd then refuses a backward after an in-place
        # change of it): the adjoint solve must use this forward's operator even
        # if the problem solved with another kappa in between
        ctx.save_for_backward(x, kappa)
        ctx.kappa_used = kd
        ctx.forward_stats = st
        problem.last_forward_stats = st
        return x

    @staticmethod
    def backward(ctx, grad_x):
        x, _ = ctx.saved_tensors
        if getattr(ctx.problem, "_kappa_ref", None) is not ctx.kappa_used:
            ctx.problem.set_kappa(ctx.kappa_used)
        gb, gk, st = ctx.problem.pcg_backward(x, grad_x.contiguous(), max_iters=ctx.max_iters, tol=ctx.tol,
                                              want_kappa=ctx.needs_input_grad[1])
        ctx.problem.last_backward_stats = st
        return gb, gk, None, None, None


def hpcg_solve(b, kappa, problem, max_iters=200, tol=1e-12):
    return HpcgSolve.apply(b, kappa, problem, max_iters, tol)
