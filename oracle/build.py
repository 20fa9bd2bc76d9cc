"""Compile the C oracle into oracle/_build/liboracle.so (gcc, -O2, no FMA contraction).

Test infrastructure: the library built here is loaded only by the tests, the smoke check and
the bench's CPU-baseline leg. The same sources also build with -fopenmp into liboracle_omp.so,
the all-core CPU baseline (row-parallel products, column-parallel solves; same results bit for bit).
"""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("oracle.c", "projection.c", "amg.c", "block_krylov.c")]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
LIB_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall", "-Wno-unknown-pragmas"]


def _build(out: str, extra, force: bool) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in SRCS):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, *extra, *SRCS, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Build liboracle.so (serial) if missing or older than its sources; return its path."""
    return _build(LIB, [], force)


def build_omp(force: bool = False) -> str | None:
    """Build liboracle_omp.so (-fopenmp); None if the compiler has no OpenMP support."""
    try:
        return _build(LIB_OMP, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        return None


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_omp(force="--force" in sys.argv))
