"""The ctypes structures of the binding have the layout of the C header: a
probe compiled from include/hpcg.h with the host C compiler prints the size of
hpcg_options and hpcg_stats and the offset of every field, which must equal
ctypes' (CPU only)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("struct_name", ["hpcg_options", "hpcg_stats"])
def test_struct_layout_matches_header(struct_name, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_2304_08232_gb300 import _lib
    st = getattr(_lib, struct_name)
    fields = [f[0] for f in st._fields_]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "hpcg.h"', "int main(void) {",
             '  printf("size %%zu\\n", sizeof(%s));' % struct_name]
    for f in fields:
        lines.append('  printf("%s %%zu\\n", offsetof(%s, %s));' % (f, struct_name, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.split() for line in out if line.strip())
    assert int(got["size"]) == ctypes.sizeof(st)
    for f in fields:
        assert int(got[f]) == getattr(st, f).offset, f
