"""Build libstokes_gb300.so in place with nvcc for sm_103a (GB300).

Compiles the translation units of csrc/ in parallel and links them into
paper_1308_4605_gb300/libstokes_gb300.so; with --bounds-check, the
bounds-checked variant libstokes_gb300_check.so (-DSTK_BOUNDS_CHECK, see
include/stokes.h).  Usage: python -m paper_1308_4605_gb300.build [--verbose]
[--ptxas-info] [--bounds-check].
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libstokes_gb300.so")
# the bounds-checked build (-DSTK_BOUNDS_CHECK): same sources, own objects
LIB_CHECK = os.path.join(HERE, "libstokes_gb300_check.so")
SOURCES = ["kernels.cu", "pair.cu", "stress.cu", "krylov.cu", "gmres.cu", "coarse.cu", "solver.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def build(verbose=False, ptxas_info=False, bounds_check=False):
    bdir = BUILD + ("_check" if bounds_check else "")
    lib = LIB_CHECK if bounds_check else LIB
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-I", os.path.join(HERE, "..", "include")]
    if bounds_check:
        flags += ["-DSTK_BOUNDS_CHECK"]
    if ptxas_info:
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [cc, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 or verbose or ptxas_info:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}")
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link failed")
    os.replace(tmp, lib)
    return lib


def build_all(verbose=False):
    """The release library and the bounds-checked one, built side by side."""
    with ThreadPoolExecutor(2) as ex:
        libs = list(ex.map(lambda bc: build(verbose=verbose, bounds_check=bc), (False, True)))
    return libs


if __name__ == "__main__":
    print(build(verbose="--verbose" in sys.argv, ptxas_info="--ptxas-info" in sys.argv,
                bounds_check="--bounds-check" in sys.argv))
