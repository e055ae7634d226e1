"""The allocation-free V-cycle against the handle-based one, through the C ABI.

hpcg_mg_vcycle_noalloc is for callers that cannot allocate device memory when
they need the preconditioner (graph capture under a strict allocator, plug-ins
inside an application that owns all device memory, real-time loops): it takes
only r and z and keeps its coarse-level vectors in a fixed array inside the
library.  Its result must match hpcg_mg_vcycle's within the FP64 tolerance of
the other parity tests, call after call, although every call reuses the same
array.  This file sorts last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from hpcg_inputs import normal
from tests.gpu_util import TOL64, dev, host, need_gpu, normwise

pytestmark = pytest.mark.gpu

HPCG_ERR_NO_WORKSPACE = 6


def _noalloc(lib, dims, levels, r, z):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.hpcg_mg_vcycle_noalloc(dims[0], dims[1], dims[2], levels, ctypes.c_void_p(r.data_ptr()),
                                      ctypes.c_void_p(z.data_ptr()), s)


def test_noalloc_vcycle_matches_handle_vcycle_on_consecutive_calls():
    need_gpu()
    from paper_2304_08232_gb300 import HpcgProblem, _lib
    lib = _lib.load()
    # consecutive calls: a second right-hand side on the same grid, then a
    # different grid, each checked against the handle-based V-cycle
    cases = [((64, 32, 48), 4, 1), ((64, 32, 48), 4, 2), ((32, 48, 16), 3, 3)]
    for dims, levels, seed in cases:
        n = int(np.prod(dims))
        r = dev(normal(n, seed))
        z = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(lib, dims, levels, r, z) == 0
        ref = HpcgProblem(*dims, levels=levels).mg_vcycle(r)
        assert normwise(host(z), host(ref)) <= TOL64


def test_noalloc_vcycle_full_size_twice():
    need_gpu()
    from paper_2304_08232_gb300 import HpcgProblem, _lib
    lib = _lib.load()
    dims, levels = (192, 192, 192), 4
    n = 192 ** 3
    prob = HpcgProblem(*dims, levels=levels)
    for seed in (0, 1):
        r = dev(normal(n, seed))
        z = torch.empty_like(r)
        assert _noalloc(lib, dims, levels, r, z) == 0
        assert normwise(host(z), host(prob.mg_vcycle(r))) <= TOL64


def test_noalloc_rejects_problems_beyond_its_array():
    need_gpu()
    from paper_2304_08232_gb300 import _lib
    lib = _lib.load()
    r = torch.zeros(8, dtype=torch.float64, device="cuda")
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    # 256^3 with 4 levels needs about 38 MB of coarse vectors: rejected on the host
    assert _noalloc(lib, (256, 256, 256), 4, r, z) == HPCG_ERR_NO_WORKSPACE
    assert _noalloc(lib, (12, 16, 16), 4, r, z) == 1   # sizes as hpcg_setup


def test_noalloc_coarse_levels_against_the_oracle():
    """The coarse levels the allocation-free V-cycle keeps in its array: each
    z_l is Listing 1 from level l on the r_l it holds, and each r_l is the
    restricted residual of the level above, point by point to rounding of the
    local magnitudes, with magnitudes spread over 80 decades between x-lines
    so that a value from the wrong place fails (the final z alone cannot show
    the coarse levels: the post-smoother recomputes the points they correct)."""
    need_gpu()
    from oracle import OracleProblem
    from paper_2304_08232_gb300 import _lib
    from tests.test_gpu_coarse_levels import _line_spread, _restriction_ok
    lib = _lib.load()
    dims, levels = (64, 32, 48), 4
    n = int(np.prod(dims))
    o = OracleProblem(*dims, levels=levels)
    eps = np.finfo(np.float64).eps
    for spread in (False, True):
        r = normal(n, 11) * (_line_spread(dims, 12) if spread else 1.0)
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        assert _noalloc(lib, dims, levels, dev(r), z) == 0
        r_prev = r
        for l in range(1, levels):
            nl = o.n(l)
            rl = torch.empty(nl, dtype=torch.float64, device="cuda")
            zl = torch.empty(nl, dtype=torch.float64, device="cuda")
            s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
            assert lib.hpcg_noalloc_level_vectors(*dims, levels, l, ctypes.c_void_p(rl.data_ptr()), ctypes.c_void_p(zl.data_ptr()),
                                                  s) == 0
            rl, zl = host(rl), host(zl)
            if not spread:
                assert normwise(zl, o.mg(rl, l)) <= TOL64, l
            zp = o.rbgs(r_prev, np.zeros(o.n(l - 1)), l - 1)
            ok, _ = _restriction_ok(o, l - 1, o.dims(l - 1), r_prev, zp, rl, 1024 * eps)
            assert ok, (spread, l)
            if spread and l < levels - 1:  # (into the 8 x 4 x 6 coarsest level the smoothed magnitudes vary too little)
                assert not _restriction_ok(o, l - 1, o.dims(l - 1), r_prev, zp, rl, 1024 * eps, shift=1)[0], l
            r_prev = rl
