"""ctypes wrapper over hpcg_oracle.c (test infrastructure; see package docstring)."""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hpcg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = None


def lib_path():
    return os.path.join(_OUT_DIR, "libhpcg_oracle.so")


def compile_source(src, out, extra=()):
    """Compiles an oracle source file (no FMA contraction, one thread) to a shared library;
    extra: more compiler flags (the sanitizer test's instrumentation)."""
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"] + list(extra) + [
        "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def source_path():
    return _SRC


def build_oracle(force=False):
    """Compile the oracle with gcc (no FMA contraction, one thread)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    return compile_source(_SRC, out)


def omp_lib_path():
    return os.path.join(_OUT_DIR, "libhpcg_oracle_omp.so")


def build_oracle_omp(force=False):
    """The same source built with -fopenmp: each SpMV's and each colour step's
    rows in one parallel loop (same bits as the plain build); the CPU
    baseline on all host cores.  Raises if the compiler has no OpenMP."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    out = omp_lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    return compile_source(_SRC, out, extra=("-fopenmp",))


def load_omp():
    """The OpenMP build, loaded (its thread count follows OMP_NUM_THREADS)."""
    return load_library(build_oracle_omp())


_d = ctypes.POINTER(ctypes.c_double)
_i = ctypes.POINTER(ctypes.c_int)
_l = ctypes.POINTER(ctypes.c_long)
_vp = ctypes.c_void_p


def load_library(path):
    """Loads a compiled oracle library and declares its functions."""
    lib = ctypes.CDLL(path)
    _declare(lib)
    return lib


def _load():
    global _LIB
    if _LIB is not None:
        return _LIB
    _LIB = load_library(build_oracle())
    return _LIB


def _declare(lib):
    lib.orc_create.restype = _vp
    lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _d]
    lib.orc_free.argtypes = [_vp]
    lib.orc_set_symmetric.argtypes = [_vp, ctypes.c_int]
    lib.orc_threads.restype = ctypes.c_int
    lib.orc_threads.argtypes = []
    lib.orc_levels.argtypes = [_vp]
    lib.orc_level_n.restype = ctypes.c_long
    lib.orc_level_n.argtypes = [_vp, ctypes.c_int]
    lib.orc_level_nnz.restype = ctypes.c_long
    lib.orc_level_nnz.argtypes = [_vp, ctypes.c_int]
    lib.orc_level_ncolors.argtypes = [_vp, ctypes.c_int]
    lib.orc_level_dims.argtypes = [_vp, ctypes.c_int, _i]
    lib.orc_export_csr.argtypes = [_vp, ctypes.c_int, _l, _i, _d]
    for f in ("orc_export_colors", "orc_export_row_nnz", "orc_export_f2c"):
        getattr(lib, f).argtypes = [_vp, ctypes.c_int, _i]
    lib.orc_export_diag.argtypes = [_vp, ctypes.c_int, _d]
    lib.orc_export_coarse.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _d]
    lib.orc_spmv.argtypes = [_vp, ctypes.c_int, _d, _d]
    lib.orc_spmv_rows.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _d, ctypes.c_long, _l, _d, _d]
    lib.orc_row_entries.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _d, ctypes.c_long, _i, _d]
    lib.orc_rbgs_color_step.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _d, _d]
    lib.orc_rbgs.argtypes = [_vp, ctypes.c_int, _d, _d]
    lib.orc_restrict.argtypes = [_vp, ctypes.c_int, _d, _d]
    lib.orc_prolong_add.argtypes = [_vp, ctypes.c_int, _d, _d]
    lib.orc_mg.argtypes = [_vp, ctypes.c_int, _d, _d]
    lib.orc_mg_apply.argtypes = [_vp, _d, _d]
    lib.orc_pcg.argtypes = [_vp, _d, _d, ctypes.c_int, ctypes.c_double, ctypes.c_int, _d]


def _pd(a):
    return a.ctypes.data_as(_d)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleProblem:
    """The HPCG hierarchy of one grid, built by the C oracle."""

    def __init__(self, nx, ny, nz, levels=4, kappa=None, symmetric=True, lib=None):
        self.lib = lib if lib is not None else _load()
        self.kappa = None if kappa is None else _f64(kappa).copy()
        self.h = self.lib.orc_create(nx, ny, nz, levels, _pd(self.kappa) if self.kappa is not None else None)
        if not self.h:
            raise ValueError("invalid grid %dx%dx%d with %d levels" % (nx, ny, nz, levels))
        self.levels = levels
        self.lib.orc_set_symmetric(self.h, 1 if symmetric else 0)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.orc_free(h)
            self.h = None

    # -- geometry and maps ------------------------------------------------
    def n(self, l=0):
        return self.lib.orc_level_n(self.h, l)

    def nnz(self, l=0):
        return self.lib.orc_level_nnz(self.h, l)

    def ncolors(self, l=0):
        return self.lib.orc_level_ncolors(self.h, l)

    def dims(self, l=0):
        d = np.zeros(3, dtype=np.int32)
        self.lib.orc_level_dims(self.h, l, d.ctypes.data_as(_i))
        return tuple(int(v) for v in d)

    def csr(self, l=0):
        import scipy.sparse as sp
        n, nnz = self.n(l), self.nnz(l)
        rp = np.zeros(n + 1, dtype=np.int64)
        col = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz, dtype=np.float64)
        self.lib.orc_export_csr(self.h, l, rp.ctypes.data_as(_l), col.ctypes.data_as(_i), _pd(val))
        return sp.csr_matrix((val, col, rp), shape=(n, n))

    def colors(self, l=0):
        out = np.zeros(self.n(l), dtype=np.int32)
        self.lib.orc_export_colors(self.h, l, out.ctypes.data_as(_i))
        return out

    def row_nnz(self, l=0):
        out = np.zeros(self.n(l), dtype=np.int32)
        self.lib.orc_export_row_nnz(self.h, l, out.ctypes.data_as(_i))
        return out

    def diag(self, l=0):
        out = np.zeros(self.n(l), dtype=np.float64)
        self.lib.orc_export_diag(self.h, l, _pd(out))
        return out

    def f2c(self, l=0):
        if l >= self.levels - 1:
            raise ValueError("the coarsest level has no injection map")
        out = np.zeros(self.n(l + 1), dtype=np.int32)
        self.lib.orc_export_f2c(self.h, l, out.ctypes.data_as(_i))
        return out

    # -- kernels ------------------------------------------------------------
    def spmv(self, x, l=0):
        x = _f64(x)
        y = np.zeros(self.n(l))
        self.lib.orc_spmv(self.h, l, _pd(x), _pd(y))
        return y

    def rhs(self):
        """HPCG right-hand side b = A * ones, so that the exact solution is ones."""
        return self.spmv(np.ones(self.n(0)))

    def rbgs_color_step(self, k, r, z, l=0):
        r = _f64(r)
        z = _f64(z).copy()
        self.lib.orc_rbgs_color_step(self.h, l, k, _pd(r), _pd(z))
        return z

    def rbgs(self, r, z, l=0):
        r = _f64(r)
        z = _f64(z).copy()
        self.lib.orc_rbgs(self.h, l, _pd(r), _pd(z))
        return z

    def restrict(self, v, l=0):
        v = _f64(v)
        out = np.zeros(self.n(l + 1))
        self.lib.orc_restrict(self.h, l, _pd(v), _pd(out))
        return out

    def prolong_add(self, zc, z, l=0):
        zc = _f64(zc)
        z = _f64(z).copy()
        self.lib.orc_prolong_add(self.h, l, _pd(zc), _pd(z))
        return z

    def mg(self, r, l=0, z0=None):
        """Listing 1 from level l; z starts from z0 (zero by default)."""
        r = _f64(r)
        z = np.zeros(self.n(l)) if z0 is None else _f64(z0).copy()
        self.lib.orc_mg(self.h, l, _pd(r), _pd(z))
        return z

    def coarse_state(self, l):
        """(r_c, z_c) that the last mg call left on coarse level l >= 1."""
        if not 1 <= l < self.levels:
            raise ValueError("coarse level out of range")
        r, z = np.zeros(self.n(l)), np.zeros(self.n(l))
        self.lib.orc_export_coarse(self.h, l, 0, _pd(r))
        self.lib.orc_export_coarse(self.h, l, 1, _pd(z))
        return r, z

    def pcg(self, b, x0=None, max_iters=50, tol=0.0, precond=True):
        b = _f64(b)
        x = np.zeros(self.n(0)) if x0 is None else _f64(x0).copy()
        hist = np.zeros(max(max_iters, 1))
        it = self.lib.orc_pcg(self.h, _pd(b), _pd(x), max_iters, tol, 1 if precond else 0, _pd(hist))
        return x, hist[:it].copy()


def spmv_rows(nx, ny, nz, rows, x, kappa=None):
    """Rows of A x generated on the fly (no CRS), for sampled checks at full size."""
    lib = _load()
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    x = _f64(x)
    y = np.zeros(len(rows))
    kp = _pd(_f64(kappa)) if kappa is not None else None
    lib.orc_spmv_rows(nx, ny, nz, kp, len(rows), rows.ctypes.data_as(_l), _pd(x), _pd(y))
    return y


def row_entries(nx, ny, nz, i, kappa=None):
    lib = _load()
    cols = np.zeros(27, dtype=np.int32)
    vals = np.zeros(27)
    kp = _pd(_f64(kappa)) if kappa is not None else None
    cnt = lib.orc_row_entries(nx, ny, nz, kp, i, cols.ctypes.data_as(_i), _pd(vals))
    return cols[:cnt].copy(), vals[:cnt].copy()


def solve_and_grad(dims, levels, kappa, b, x_target, tol=1e-14, max_iters=500):
    """Differentiable form: forward x = A(kappa)^{-1} b, loss 0.5 ||x - x_t||^2,
    adjoint lambda = A^{-1} (x - x_t) (A is symmetric), grad_b = lambda,
    grad_kappa_i = -lambda_i x_i (the diagonal of -lambda x^T, since
    dA/dkappa_i = e_i e_i^T).  Both solves are the oracle's MG-PCG."""
    p = OracleProblem(*dims, levels=levels, kappa=kappa)
    x, _ = p.pcg(b, max_iters=max_iters, tol=tol)
    g = x - np.asarray(x_target, dtype=np.float64)
    lam, _ = p.pcg(g, max_iters=max_iters, tol=tol)
    loss = 0.5 * float(g @ g)
    return x, loss, lam, -lam * x
