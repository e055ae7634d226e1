"""FP64 CPU oracle for the HPCG-on-GraphBLAS hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it.  The arithmetic lives in ``hpcg_oracle.c`` (plain C,
single thread, ``-ffp-contract=off``); this module only builds it, loads it with
ctypes and marshals numpy arrays.

Functions follow the paper section by section (Scolari & Yzelman, "Effective
implementation of the High Performance Conjugate Gradient benchmark on
GraphBLAS"): input generation (Sec. II-B), CRS operator with separate A_diag
(Sec. III-A), greedy colouring (Sec. III-A), red-black Gauss-Seidel colour
steps (Listings 2 and 3), straight injection and its transpose (Sec. II-F,
III-B), the MG V-cycle (Listing 1) and preconditioned CG (Sec. II-C).

Parity status: every function is pinned by a test in tests/test_oracle_*.py
against closed forms, brute force, dense textbook routines or dense direct
solves; the exact per-iteration residual history is pinned only through
those properties (the paper prints no worked example).
"""
from .oracle import (OracleProblem, build_oracle, build_oracle_omp, load_omp, spmv_rows, lib_path,  # noqa: F401
                     solve_and_grad)
