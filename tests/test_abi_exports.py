"""The C-ABI library builds, loads and exports every entry point that
include/hpcg.h declares (CPU only: no compute call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hpcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hpcg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_08232_gb300 import _lib
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 25
    for name in names:
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol():
    from paper_2304_08232_gb300._lib import SIGNATURES
    assert set(_declared()) == set(SIGNATURES)


def test_host_only_calls(lib):
    from paper_2304_08232_gb300._lib import hpcg_options
    h = ctypes.c_void_p()
    assert lib.hpcg_setup(16, 16, 16, 4, ctypes.byref(h)) == 0
    nb = ctypes.c_size_t()
    assert lib.hpcg_workspace_bytes(h, ctypes.byref(nb)) == 0
    assert nb.value > 4 * 4096 * 8
    d = (ctypes.c_int * 3)()
    assert lib.hpcg_level_dims(h, 3, d) == 0 and tuple(d) == (2, 2, 2)
    assert lib.hpcg_level_dims(h, 4, d) == 1
    # invalid sizes are rejected on the host
    bad = ctypes.c_void_p()
    assert lib.hpcg_setup(12, 16, 16, 4, ctypes.byref(bad)) == 1   # 12 not divisible by 8
    assert lib.hpcg_setup(8, 8, 8, 4, ctypes.byref(bad)) == 1      # coarsest edge 1
    assert lib.hpcg_setup(16, 16, 16, 0, ctypes.byref(bad)) == 1
    assert lib.hpcg_setup(16, 16, 16, 4, None) == 1
    opt = hpcg_options()
    assert lib.hpcg_options_default(ctypes.byref(opt), 8, 8, 8) == 0
    assert (opt.levels, opt.pre_sweeps, opt.post_sweeps, opt.symmetric) == (4, 1, 1, 1)
    dims = (ctypes.c_int * 6)(32, 48, 64, 96, 80, 32)
    hb = ctypes.c_void_p()
    assert lib.hpcg_setup_batch(2, dims, 4, 0, ctypes.byref(hb)) == 0
    offs = (ctypes.c_long * 3)()
    assert lib.hpcg_batch_offsets(hb, offs) == 0
    assert list(offs) == [0, 32 * 48 * 64, 32 * 48 * 64 + 96 * 80 * 32]
    assert lib.hpcg_strerror(4) == b"tolerance not reached within max_iters"
    # handles without a bound workspace are freed without touching the device
    assert lib.hpcg_destroy(h) == 0
    assert lib.hpcg_destroy(hb) == 0
