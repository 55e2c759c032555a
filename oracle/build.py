"""Build the FP64 oracle (plain C, gcc) into oracle/_build/liboracle.so.

Test infrastructure only.  Flags: -O2, OpenMP for the batch drivers, and -ffp-contract=off so
that x86-64 and AArch64 builds round identically (no fused multiply-adds).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["chart.c", "hermite.c", "sh.c", "bake.c", "procedural.c", "query.c", "adjoint.c", "raycast.c", "mip.c", "recon.c"]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["oracle.h"]
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in deps)


def build(verbose: bool = False) -> str:
    if not needs_build():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-Wall", "-Wno-unused-function", "-o", tmp] + [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
