"""The oracle under the host compiler's address and undefined-behaviour
sanitizers: every pin of tests/test_oracle_mutants.py runs on an instrumented
build (out-of-bounds accesses, use after free, signed overflow, misaligned or
null accesses abort the run), CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, %r)
from oracle.oracle import load_library
from tests.test_oracle_mutants import _pins
res = _pins(load_library(%r))
failed = [name for name, ok in res if not ok]
print("pins", len(res), "failed", failed)
sys.exit(1 if failed or not res else 0)
"""


FLAGS = ["-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined", "-fno-sanitize-recover=all"]


def _run_pins(src, tmp_path, name):
    from oracle.oracle import compile_source
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not asan or not os.path.exists(asan):
        pytest.skip("no libasan for the host compiler")
    lib = str(tmp_path / name)
    compile_source(src, lib, extra=FLAGS)
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1:verify_asan_link_order=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    return subprocess.run([sys.executable, "-c", SCRIPT % (ROOT, lib)], env=env, capture_output=True, text=True, timeout=900)


def test_oracle_pins_clean_under_asan_and_ubsan(tmp_path):
    from oracle.oracle import source_path
    r = _run_pins(source_path(), tmp_path, "liboracle_sanitized.so")
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert "failed []" in r.stdout


def test_sanitizer_catches_a_planted_overrun(tmp_path):
    """The harness is live: the injection loop run one coarse row too far reads
    past the end of the map and the instrumented run aborts."""
    from oracle.oracle import source_path
    src = open(source_path()).read()
    old = "  for (long c = 0; c < nc; ++c) rc[c] = v[F->f2c[c]];"
    assert old in src
    bad = tmp_path / "oracle_overrun.c"
    bad.write_text(src.replace(old, "  for (long c = 0; c <= nc; ++c) rc[c] = v[F->f2c[c]];"))
    r = _run_pins(str(bad), tmp_path, "liboracle_overrun.so")
    assert r.returncode != 0 and "AddressSanitizer" in r.stderr
