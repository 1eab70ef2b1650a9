"""Build the oracle's shared library (plain C, FP64) with gcc.

TEST INFRASTRUCTURE ONLY: the oracle checks the CUDA path; nothing on the
product path may load it.  No floating-point contraction and no fast-math, so
its FP64 results are the same on x86-64 and aarch64 hosts.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["or_philox.c", "or_math.c", "or_batchrng.c", "or_gibbs.c", "or_lda.c"]
LIB = os.path.join(HERE, "liboracle.so")
CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-pthread",
          "-Wall", "-Wextra", "-Wno-unused-parameter"]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["oracle.h", "or_internal.h"]
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in deps)


def build(force: bool = False) -> str:
    if force or needs_build():
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", *CFLAGS, "-shared", "-o", tmp, *[os.path.join(HERE, s) for s in SOURCES], "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
