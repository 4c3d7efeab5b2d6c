"""Compile the oracle's plain-C sweep (test infrastructure only).

    python -m oracle.build        # writes oracle/_oracle_sweep.so

Plain gcc, no vendor libraries, portable flags (the same source builds on
x86_64 and aarch64 hosts).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sweep.c")
LIB = os.path.join(HERE, "_oracle_sweep.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-fno-fast-math",
           "-ffp-contract=off", SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
