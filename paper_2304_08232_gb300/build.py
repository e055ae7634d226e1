"""Builds the in-tree CUDA library libhpcg_gb300.so for sm_103a with nvcc.

Translation units are compiled in parallel, then linked into one shared
library exporting the C ABI of include/hpcg.h.  The output goes to
paper_2304_08232_gb300/_build/ (git-ignored).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libhpcg_gb300.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def lib_path():
    return os.path.join(OUT_DIR, LIB_NAME)


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra=(), out_dir=None, lib_name=None):
    nvcc = os.environ.get("NVCC", "nvcc")
    out_dir = out_dir or OUT_DIR
    os.makedirs(out_dir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "hpcg.h"))
    srcs = sources()
    objs = []
    procs = []
    for src in srcs:
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers + [os.path.abspath(__file__)]):
            cmd = [nvcc] + ARCH + FLAGS + list(extra) + ["-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for: %s" % ", ".join(failed))
    out = os.path.join(out_dir, lib_name or LIB_NAME)
    if force or _stale(out, objs):
        tmp = out + ".tmp%d" % os.getpid()
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    return out


def build_checked(force=False, verbose=False):
    """The bounds-checking build (-DHPCG_BOUNDS_CHECK) into its own folder:
    every index range the default FP64 path touches is checked against its
    array's extent, a miss recorded and skipped (hpcg_bounds_status)."""
    return build(force=force, verbose=verbose, extra=("-DHPCG_BOUNDS_CHECK",), out_dir=os.path.join(HERE, "_build_bc"),
                 lib_name="libhpcg_gb300_bc.so")


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, extra=[a for a in sys.argv[1:] if a.startswith("-X")]))
