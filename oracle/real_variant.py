"""ORACLE -- test infrastructure only (see oracle/__init__.py).

Real-arithmetic variant of Algorithm 3 for real A_j and real B: the real Schur
form A_j = Q_j T_j Q_j^T (Q_j orthogonal, T_j quasi-upper-triangular with 2 x 2
diagonal blocks for complex-conjugate eigenvalue pairs) replaces the complex
Schur form of Section 2, so every tensor stays real.

  setup    A_j = Q_j T_j Q_j^T, scipy's real Schur (a library primitive);
  forward  C = Q_N^T (x)_N ( ... (Q_1^T (x)_1 B))     (Eq. (CUNU2U1B) with U_j = Q_j);
  sweep    Eq. (yi1i2iN) with the entries of one diagonal block of every mode
           solved together: for a block multi-index beta (a 1 x 1 or 2 x 2 block
           per mode, visited in the nesting order of Algorithm 1), the entries
           i of the box beta satisfy
               sum_j sum_{k in beta_j} T_j[i_j, k] Y[..k..]
                   = C[i] - sum_j sum_{k after beta_j} T_j[i_j, k] Y[..k..],
           a dense system of prod_j |beta_j| <= 2^N unknowns, solved by
           numpy.linalg.solve (a library primitive); with only 1 x 1 blocks it
           is the division of Eq. (yi1i2iN);
  back     X = Q_N (x)_N ( ... (Q_1 (x)_1 Y))          (Eq. (XUNU2U1Y)).

Pure-Python loops over the block multi-indices: small inputs only.
"""
from __future__ import annotations

import itertools
from typing import List, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg

from .bartels_stewart import mode_product


def real_schur_factors(A: Sequence[np.ndarray]):
    """[(Q_j or None, T_j)] with A_j = Q_j T_j Q_j^T, T_j quasi-upper-triangular."""
    out = []
    for Aj in A:
        Aj = np.asarray(Aj, dtype=np.float64)
        if Aj.shape == (1, 1):
            out.append((None, Aj.copy()))
        else:
            T, Q = scipy.linalg.schur(Aj, output="real")
            out.append((Q, T))
    return out


def diagonal_blocks(T: np.ndarray) -> List[Tuple[int, int]]:
    """(start, size) of the diagonal blocks of a quasi-upper-triangular T: a
    nonzero T[k+1, k] couples k and k+1 into one 2 x 2 block."""
    n = T.shape[0]
    out, k = [], 0
    while k < n:
        s = 2 if (k + 1 < n and T[k + 1, k] != 0.0) else 1
        out.append((k, s))
        k += s
    return out


def forward_transform_real(Q: Sequence[Optional[np.ndarray]], B: np.ndarray) -> np.ndarray:
    """C = Q_N^T (x)_N ( ... (Q_1^T (x)_1 B))."""
    C = np.array(B, dtype=np.float64, order="F", copy=True)
    for j, Qj in enumerate(Q):
        if Qj is not None:
            C = mode_product(Qj.T, C, j)
    return C


def back_transform_real(Q: Sequence[Optional[np.ndarray]], Y: np.ndarray) -> np.ndarray:
    """X = Q_N (x)_N ( ... (Q_1 (x)_1 Y))."""
    X = np.array(Y, dtype=np.float64, order="F", copy=True)
    for j, Qj in enumerate(Q):
        if Qj is not None:
            X = mode_product(Qj, X, j)
    return X


def quasi_triangular_sweep(T: Sequence[np.ndarray], C: np.ndarray) -> np.ndarray:
    """Y with sum_j T_j (x)_j Y = C for quasi-upper-triangular T_j (real)."""
    N = len(T)
    n = [t.shape[0] for t in T]
    blocks = [diagonal_blocks(np.asarray(t)) for t in T]
    Y = np.array(C, dtype=np.float64, order="F", copy=True)
    extra = Y.shape[N:]
    for tail in itertools.product(*[range(e) for e in extra]):
        # block multi-indices, last mode outermost, each mode from its last block
        for rev in itertools.product(*[list(reversed(b)) for b in reversed(blocks)]):
            beta = tuple(reversed(rev))                      # ((start, size), ...)
            box = list(itertools.product(*[range(s, s + z) for s, z in beta]))
            pos = {ii: p for p, ii in enumerate(box)}
            m = len(box)
            M = np.zeros((m, m))
            rhs = np.zeros(m)
            for p, ii in enumerate(box):
                num = Y[ii + tail]
                for j in range(N):
                    s, z = beta[j]
                    for k in range(s, s + z):                # inside the block: unknowns
                        kk = ii[:j] + (k,) + ii[j + 1:]
                        M[p, pos[kk]] += T[j][ii[j], k]
                    for k in range(s + z, n[j]):             # later blocks: solved
                        kk = ii[:j] + (k,) + ii[j + 1:]
                        num -= T[j][ii[j], k] * Y[kk + tail]
                rhs[p] = num
            y = np.linalg.solve(M, rhs)
            for p, ii in enumerate(box):
                Y[ii + tail] = y[p]
    return Y


def solve_real_with_factors(factors, B: np.ndarray) -> np.ndarray:
    Q = [f[0] for f in factors]
    T = [f[1] for f in factors]
    return back_transform_real(Q, quasi_triangular_sweep(T, forward_transform_real(Q, B)))


def solve_real(A: Sequence[np.ndarray], B: np.ndarray) -> np.ndarray:
    """X with sum_j A_j (x)_j X = B for real A_j and B, in real arithmetic."""
    return solve_real_with_factors(real_schur_factors(A), B)
