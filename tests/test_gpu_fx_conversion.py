"""The int64 -> FP64 conversion that the fixed-point sums and the
block-floating-point V-cycle build on the integer pipe (fx_to_double), bit for
bit against CUDA's round-to-nearest __ll2double_rn scaled exactly by the same
power of two: ties to even, the mantissa carry into the exponent, values near
2^62, both signs, zero, and the exponent bounds the kernels use."""
import ctypes

import numpy as np
import pytest
import torch

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

E_MIN, E_MAX = 64, 2000


def _cases():
    q = []
    for k in range(53, 63):  # lengths where the last kept bit and the dropped bits meet
        b = 1 << k
        drop = 1 << (k - 52)  # value of one unit in the last place at this length
        half = drop >> 1
        q += [b, b + half, b + drop + half, b + half + 1, b + half - 1,  # ties to even (down, up) and near-ties
              2 * b - 1, 2 * b - half, 2 * b - half - 1,                  # mantissa all ones: carry into the exponent
              b + drop, b + 3 * half]
    q += [0, 1, 2, 3, (1 << 53) - 1, (1 << 62) + (1 << 61), (1 << 63) - 1, (1 << 63) - 512, (1 << 63) - 1024]
    rng = np.random.default_rng(7)
    for bits in range(1, 63):
        q += [int(v) for v in rng.integers(1 << (bits - 1), 1 << bits, size=8, dtype=np.int64)]
    q = np.array(q + [-v for v in q], dtype=np.int64)
    return q


@pytest.mark.parametrize("E", [E_MIN, E_MIN + 1, 1080, 1081, 1500, E_MAX - 1, E_MAX])
def test_fx_to_double_matches_cuda_conversion(E):
    need_gpu()
    from paper_2304_08232_gb300 import _lib
    lib = _lib.load()
    q = torch.as_tensor(_cases(), device="cuda")
    e = torch.full(q.shape, E, dtype=torch.int32, device="cuda")
    out = torch.empty(q.shape, dtype=torch.float64, device="cuda")
    ref = torch.empty_like(out)
    rc = lib.hpcg_fx_to_double_check(q.numel(), ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(e.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ref.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    o, r = out.cpu().numpy(), ref.cpu().numpy()
    assert np.array_equal(o.view(np.int64), r.view(np.int64)), np.nonzero(o != r)
    # and the host's exact arithmetic agrees on the values where the power of two keeps them normal
    qs = _cases()
    host = np.array([float(int(v)) for v in qs]) * np.ldexp(1.0, E - 1080)
    fin = np.isfinite(host) & (np.abs(host) >= np.finfo(np.float64).tiny) | (qs == 0)
    assert np.array_equal(o[fin].view(np.int64), host[fin].view(np.int64))
