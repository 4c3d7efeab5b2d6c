"""Writes stored expected values from the oracle only (no CUDA code involved).

    python tests/golden/make_golden.py

cube_n8_N3_X.txt: the solution X of the N=3, n=8 workload (seed 0), column-major,
one entry per line as "re im" with 17 significant digits.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import sylv_inputs as si  # noqa: E402


def main():
    p = si.cube_n8_N3()
    X = oracle.solve(p.A, p.B)
    flat = X.reshape(-1, order="F")
    with open(os.path.join(HERE, "cube_n8_N3_X.txt"), "w") as f:
        f.write("# oracle solution of the N=3, n=8 workload (seed 0); column-major; re im\n")
        for z in flat:
            f.write(f"{z.real:.17e} {z.imag:.17e}\n")


if __name__ == "__main__":
    main()
