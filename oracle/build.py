"""Compile the oracle's plain-C parts (test infrastructure only).

    python -m oracle.build        # writes oracle/_oracle_sweep.so

sweep.c (the sequential sweep of Algorithm 3) and modeprod.c (the mode-j
product, OpenMP across independent fibres) in one library.  Plain gcc, no
vendor libraries, portable flags (the same sources build on x86_64 and aarch64
hosts); without OpenMP the fibre loop runs on one thread.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "sweep.c"), os.path.join(HERE, "modeprod.c")]
LIB = os.path.join(HERE, "_oracle_sweep.so")


def build(force: bool = False) -> str:
    deps = SRCS + [os.path.abspath(__file__)]
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(s) for s in deps)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O3", "-fPIC", "-shared", "-std=c99", "-fno-fast-math",
            "-ffp-contract=off"]
    r = subprocess.run(base + ["-fopenmp", *SRCS, "-o", tmp], capture_output=True)
    if r.returncode != 0:
        subprocess.run(base + [*SRCS, "-o", tmp], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
