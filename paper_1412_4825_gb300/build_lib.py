"""Build libbrng.so (the CUDA library behind include/brng.h) for sm_103a.

nvcc compiles each translation unit in parallel into _build/ and links the
shared library next to this file, where the ctypes binding loads it.  No
fast-math: the FP32 transforms use the accurate logf/sincospif/sqrtf, and the
FP64 parts are written with explicit round-to-nearest intrinsics.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libbrng.so")
SOURCES = ["brng_api.cu", "brng_bulk.cu", "brng_dirichlet.cu", "brng_gibbs.cu", "brng_static.cu",
           "brng_batch.cu", "brng_serve.cu", "brng_gibbs_pc.cu", "brng_lda_full.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for p in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if p and os.path.exists(p):
            return p
    raise RuntimeError("nvcc not found: libbrng.so cannot be built")


def _deps():
    out = [os.path.join(INCLUDE, "brng.h")]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h", ".cu"))]
    return out


# the checked build (-DBRNG_DEBUG): protocol checks counted on the device
# (csrc/brng_debug.cuh), same results; built on demand by its test
LIB_DEBUG = os.path.join(PKG, "libbrng_debug.so")


def needs_build(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), debug: bool = False) -> str:
    lib_path = LIB_DEBUG if debug else LIB
    if not (force or needs_build(lib_path)):
        return lib_path
    build_dir = BUILD + ("_debug" if debug else "")
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    if debug:
        extra = (*extra, "-DBRNG_DEBUG")

    def compile_one(src):
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            sys.stdout.write(log)
    tmp = lib_path + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    extra = ["-Xptxas", "-v"] if "-v" in sys.argv else []
    print(build(force=True, verbose=bool(extra), extra=extra))
