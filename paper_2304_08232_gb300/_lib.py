"""ctypes declarations of the C ABI in include/hpcg.h.

Loading fails loudly (ImportError) when the CUDA library has not been built:
there is no CPU fallback anywhere in this package.
"""
import ctypes
import os

from . import build as _build

_vp = ctypes.c_void_p
_i = ctypes.c_int
_l = ctypes.c_long
_d = ctypes.c_double


class hpcg_options(ctypes.Structure):
    _fields_ = [("nx", _i), ("ny", _i), ("nz", _i), ("levels", _i), ("precision", _i), ("pre_sweeps", _i),
                ("post_sweeps", _i), ("symmetric", _i), ("check_every", _i), ("max_rhs", _i), ("autotune", _i),
                ("fixed_point", _i), ("pdl", _i), ("persistent", _i), ("block_fp", _i), ("cluster_tail", _i),
                ("restart_every", _i), ("bfp_split", _i), ("fuse_planes", _i)]


class hpcg_stats(ctypes.Structure):
    _fields_ = [("iters", _i), ("restarts", _i), ("converged", _i), ("status", _i), ("rel_res", _d),
                ("history", ctypes.POINTER(_d)), ("history_cap", _i)]


# name -> (restype, argtypes)
SIGNATURES = {
    "hpcg_options_default": (_i, [ctypes.POINTER(hpcg_options), _i, _i, _i]),
    "hpcg_setup": (_i, [_i, _i, _i, _i, ctypes.POINTER(_vp)]),
    "hpcg_setup_ex": (_i, [ctypes.POINTER(hpcg_options), _vp, ctypes.POINTER(_vp)]),
    "hpcg_set_kappa": (_i, [_vp, _vp, _vp]),
    "hpcg_destroy": (_i, [_vp]),
    "hpcg_workspace_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "hpcg_bind_workspace": (_i, [_vp, _vp, ctypes.c_size_t]),
    "hpcg_level_dims": (_i, [_vp, _i, ctypes.POINTER(_i)]),
    "hpcg_get_colors": (_i, [_vp, _i, _vp, _vp]),
    "hpcg_get_f2c": (_i, [_vp, _i, _vp, _vp]),
    "hpcg_get_row_nnz": (_i, [_vp, _i, _vp, _vp]),
    "hpcg_get_rhs": (_i, [_vp, _vp, _vp]),
    "hpcg_spmv": (_i, [_vp, _i, _vp, _vp, _vp]),
    "hpcg_rbgs_color": (_i, [_vp, _i, _i, _vp, _vp, _vp]),
    "hpcg_rbgs": (_i, [_vp, _i, _vp, _vp, _vp]),
    "hpcg_restrict_residual": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
    "hpcg_prolong_add": (_i, [_vp, _i, _vp, _vp, _vp]),
    "hpcg_mg_vcycle": (_i, [_vp, _vp, _vp, _vp]),
    "hpcg_mg_stage": (_i, [_vp, _i, _i, _vp, _vp, _vp]),
    "hpcg_get_level_vectors": (_i, [_vp, _i, _vp, _vp, _vp]),
    "hpcg_set_level_vectors": (_i, [_vp, _i, _vp, _vp, _vp]),
    "hpcg_dot": (_i, [_vp, _l, _vp, _vp, _vp, _vp]),
    "hpcg_waxpby": (_i, [_vp, _l, _d, _vp, _d, _vp, _vp, _vp]),
    "hpcg_pcg_solve": (_i, [_vp, _vp, _vp, _i, _d, ctypes.POINTER(hpcg_stats), _vp]),
    "hpcg_pcg_backward": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _d, ctypes.POINTER(hpcg_stats), _vp]),
    "hpcg_pcg_solve_multi": (_i, [_vp, _i, _vp, _vp, _i, _d, ctypes.POINTER(hpcg_stats), _vp]),
    "hpcg_setup_batch": (_i, [_i, ctypes.POINTER(_i), _i, _i, ctypes.POINTER(_vp)]),
    "hpcg_batch_offsets": (_i, [_vp, ctypes.POINTER(_l)]),
    "hpcg_pcg_solve_batch": (_i, [_vp, _vp, _vp, _i, _d, ctypes.POINTER(hpcg_stats), _vp]),
    "hpcg_mg_vcycle_noalloc": (_i, [_i, _i, _i, _i, _vp, _vp, _vp]),
    "hpcg_noalloc_level_vectors": (_i, [_i, _i, _i, _i, _i, _vp, _vp, _vp]),
    "hpcg_autotune": (_i, [_vp, ctypes.POINTER(_i), _vp]),
    "hpcg_set_launch_shapes": (_i, [_vp, ctypes.POINTER(_i)]),
    "hpcg_set_wait_limit": (_i, [_vp, ctypes.c_longlong]),
    "hpcg_profile_iteration": (_i, [_vp, _vp, _vp, ctypes.POINTER(_d), _i, _vp]),
    "hpcg_device_status": (_i, [_vp, ctypes.POINTER(_i)]),
    "hpcg_persistent_levels": (_i, [_vp, ctypes.POINTER(_i)]),
    "hpcg_ell_setup": (_i, [_i, _i, _i, _i, _i, _i, _i, ctypes.POINTER(_vp)]),
    "hpcg_ell_destroy": (_i, [_vp]),
    "hpcg_ell_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "hpcg_ell_level_info": (_i, [_vp, _i, ctypes.POINTER(_l)]),
    "hpcg_ell_permutation": (_i, [_vp, _i, _vp, _vp]),
    "hpcg_ell_matrix": (_i, [_vp, _i, _vp, _vp, _vp]),
    "hpcg_ell_permute": (_i, [_vp, _i, _i, _vp, _vp, _vp]),
    "hpcg_ell_spmv": (_i, [_vp, _i, _vp, _vp, _vp]),
    "hpcg_ell_rbgs_color": (_i, [_vp, _i, _i, _vp, _vp, _vp]),
    "hpcg_ell_rbgs": (_i, [_vp, _i, _vp, _vp, _vp]),
    "hpcg_ell_mg_vcycle": (_i, [_vp, _vp, _vp, _vp]),
    "hpcg_ell_pcg_solve": (_i, [_vp, _vp, _vp, _i, _d, ctypes.POINTER(hpcg_stats), _vp]),
    "hpcg_split_setup": (_i, [_i, _i, _i, _i, _i, ctypes.POINTER(_vp)]),
    "hpcg_split_destroy": (_i, [_vp]),
    "hpcg_split_info": (_i, [_vp, _i, _i, ctypes.POINTER(_l)]),
    "hpcg_split_exchange_count": (_i, [_vp, ctypes.POINTER(_l), ctypes.POINTER(_l)]),
    "hpcg_split_spmv": (_i, [_vp, _i, _vp, _vp, _vp]),
    "hpcg_split_rbgs": (_i, [_vp, _i, _vp, _vp, _vp]),
    "hpcg_split_mg_vcycle": (_i, [_vp, _vp, _vp, _vp]),
    "hpcg_split_pcg_solve": (_i, [_vp, _vp, _vp, _i, _d, ctypes.POINTER(hpcg_stats), _vp]),
    "hpcg_probe_fp64_rate": (_i, [_i, _i, _vp, ctypes.POINTER(_d), ctypes.POINTER(_d), _vp]),
    "hpcg_fx_to_double_check": (_i, [_l, _vp, _vp, _vp, _vp, _vp]),
    "hpcg_bounds_status": (_i, [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), _i]),
    "hpcg_strerror": (ctypes.c_char_p, [_i]),
    "hpcg_last_cuda_error": (ctypes.c_char_p, []),
    "hpcg_launch_count": (_l, []),
}

HPCG_OK = 0
HPCG_ERR_NOT_CONVERGED = 4
FP64, MIXED = 0, 1
STAGE_PRE, STAGE_REFINE, STAGE_POST = 0, 1, 2

_LIB = None


def _open(path):
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(path=None):
    """Loads the built library (no build here); raises ImportError if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.lib_path()
    if not os.path.exists(path):
        raise ImportError("CUDA library %s is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    _LIB = _open(path)
    return _LIB


_LIB_CHECKED = None


def load_checked():
    """The bounds-checking build of the library (built on first use with
    build.build_checked; a second library beside the normal one)."""
    global _LIB_CHECKED
    if _LIB_CHECKED is None:
        _LIB_CHECKED = _open(_build.build_checked())
    return _LIB_CHECKED


class HpcgError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.hpcg_strerror(status).decode()
        if status == 2:
            msg += " (" + lib.hpcg_last_cuda_error().decode() + ")"
        super().__init__("%s: %s [status %d]" % (where, msg, status))
        self.status = status


def check(status, where, allow=()):
    if status != HPCG_OK and status not in allow:
        raise HpcgError(status, where)
    return status
