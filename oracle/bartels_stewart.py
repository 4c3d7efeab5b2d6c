"""ORACLE -- test infrastructure only (see oracle/__init__.py).

Plain FP64 restatement of the method of Cuesta & de la Hoz, arXiv 2412.15840:

  problem      sum_j A_j (x)_j X = B,  [A (x)_j X]_{..i_j..} = sum_k a_{i_j k} x_{..k..}
               (Section 1, Eq. (sylvesterND));
  setup        A_j = U_j T_j U_j^*, complex Schur (Section 2); a singleton mode
               keeps T_j = A_j and has no U_j (Section 4);
  forward      C = U_N^* (x)_N ( ... (U_1^* (x)_1 B))      (Eq. (CUNU2U1B));
  sweep        Eq. (yi1i2iN) in the order of Algorithm 3     (oracle/sweep.c);
  back         X = U_N (x)_N ( ... (U_1 (x)_1 Y))          (Eq. (XUNU2U1Y)).

Tensors are numpy arrays indexed logically as (i_1, ..., i_N[, rhs]), stored
column-major (Fortran order), as in Eq. (index).  Any trailing axes beyond the
N modes are independent right-hand sides.  A library matrix product
(numpy.tensordot) serves as the mode-j product step; nothing is blocked, fused
or reordered beyond the paper's own order.
"""
from __future__ import annotations

import ctypes
import itertools
import time
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_sweep.restype = ctypes.c_int
        lib.oracle_sweep.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]
        lib.oracle_mode_product.restype = ctypes.c_int
        lib.oracle_mode_product.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_set_threads.restype = None
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_counter_order.restype = ctypes.c_int
        lib.oracle_counter_order.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                             ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        _LIB = lib
    return _LIB


# ----------------------------------------------------------------------------
# Index conventions (Section 2.2, Eq. (index) and Algorithm 2)
# ----------------------------------------------------------------------------

def linear_index(ii: Sequence[int], n: Sequence[int]) -> int:
    """1-based column-major index of the 1-based multi-index ii (Eq. (index))."""
    index, stride = 1, 1
    for i, nj in zip(ii, n):
        index += (i - 1) * stride
        stride *= nj
    return index


def counter_order(n: Sequence[int], count: Optional[int] = None) -> List[Tuple[int, ...]]:
    """First `count` tuples produced by the mixed-radix counter of Algorithm 2."""
    N = len(n)
    total = int(np.prod(n))
    count = total if count is None else count
    nn = (ctypes.c_int64 * N)(*n)
    out = (ctypes.c_int64 * (count * N))()
    rc = _lib().oracle_counter_order(N, nn, count, out)
    if rc != 0:
        raise RuntimeError("oracle_counter_order failed")
    flat = list(out)
    return [tuple(flat[t * N:(t + 1) * N]) for t in range(count)]


# ----------------------------------------------------------------------------
# Mode-j product and the operator (Section 1)
# ----------------------------------------------------------------------------

def mode_product(M: np.ndarray, X: np.ndarray, j: int) -> np.ndarray:
    """[M (x)_j X]_{..i..} = sum_k M[i, k] X[..k..] along axis j (0-based).

    X (column-major) is viewed as (L, n_j, R) with L = prod_{m<j} n_m and
    R = prod_{m>j} n_m, so that out[l, i, r] = sum_k M[i, k] X[l, k, r]:
    complex data in oracle/modeprod.c (plain loops, k ascending), real data
    (the real-arithmetic variant) as one library matrix product per slice over
    the shorter of L and R."""
    if M.shape == (1, 1):
        return M[0, 0] * X                                  # scalar case, Section 4
    X = np.asfortranarray(X)
    shp = X.shape
    L = int(np.prod(shp[:j], dtype=np.int64))
    n = int(shp[j])
    R = int(np.prod(shp[j + 1:], dtype=np.int64))
    if np.iscomplexobj(M) or np.iscomplexobj(X):
        Mc = np.asfortranarray(M, dtype=np.complex128)
        Xc = np.asfortranarray(X, dtype=np.complex128)
        out = np.empty(shp, dtype=np.complex128, order="F")
        if _lib().oracle_mode_product(L, n, R, Mc.ctypes.data, Xc.ctypes.data,
                                      out.ctypes.data) != 0:
            raise RuntimeError("oracle_mode_product: bad arguments")
        return out
    X3 = X.reshape((L, n, R), order="F")
    out = np.empty((L, n, R), dtype=np.result_type(M, X), order="F")
    if L >= R:
        for r in range(R):
            out[:, :, r] = X3[:, :, r] @ M.T                # out[l, i] = sum_k X[l, k] M[i, k]
    else:
        for l in range(L):
            out[l, :, :] = M @ X3[l, :, :]                  # out[i, r] = sum_k M[i, k] X[k, r]
    return out.reshape(shp, order="F")


def apply_operator(A: Sequence[np.ndarray], X: np.ndarray) -> np.ndarray:
    """sum_j A_j (x)_j X over the first len(A) axes of X."""
    acc = np.zeros_like(X, order="F")
    for j, Aj in enumerate(A):
        acc += mode_product(Aj, X, j)
    return acc


def residual(A: Sequence[np.ndarray], X: np.ndarray, B: np.ndarray) -> np.ndarray:
    return B - apply_operator(A, X)


# ----------------------------------------------------------------------------
# Setup: complex Schur factors (Section 2; Section 4 for singleton modes)
# ----------------------------------------------------------------------------

def schur_factors(A: Sequence[np.ndarray], sort=None):
    """[(U_j or None, T_j)] with A_j = U_j T_j U_j^*, T_j upper triangular."""
    out = []
    for Aj in A:
        Aj = np.asarray(Aj, dtype=np.complex128)
        if Aj.shape == (1, 1):
            out.append((None, Aj.copy()))
        else:
            if sort is None:
                T, U = scipy.linalg.schur(Aj, output="complex")
            else:
                T, U, _ = scipy.linalg.schur(Aj, output="complex", sort=sort)
            out.append((U, np.triu(T)))
    return out


# ----------------------------------------------------------------------------
# The three phases
# ----------------------------------------------------------------------------

def forward_transform(U: Sequence[Optional[np.ndarray]], B: np.ndarray) -> np.ndarray:
    """C = U_N^* (x)_N ( ... (U_1^* (x)_1 B)),  Eq. (CUNU2U1B)."""
    C = np.array(B, dtype=np.complex128, order="F", copy=True)
    for j, Uj in enumerate(U):
        if Uj is not None:
            C = mode_product(Uj.conj().T, C, j)
    return C


def back_transform(U: Sequence[Optional[np.ndarray]], Y: np.ndarray) -> np.ndarray:
    """X = U_N (x)_N ( ... (U_1 (x)_1 Y)),  Eq. (XUNU2U1Y)."""
    X = np.array(Y, dtype=np.complex128, order="F", copy=True)
    for j, Uj in enumerate(U):
        if Uj is not None:
            X = mode_product(Uj, X, j)
    return X


def triangular_sweep(T: Sequence[np.ndarray], C: np.ndarray) -> np.ndarray:
    """Y with sum_j T_j (x)_j Y = C, by the sequential sweep of Algorithm 3.

    Axes beyond len(T) are independent right-hand sides, each swept on its own.
    """
    N = len(T)
    n = [int(t.shape[0]) for t in T]
    Y = np.array(C, dtype=np.complex128, order="F", copy=True)
    lead = int(np.prod(n))
    rest = int(Y.size // lead) if lead else 0
    flat = Y.reshape(lead, rest, order="F")                 # a view (Fortran order)
    Tc = [np.asfortranarray(t, dtype=np.complex128) for t in T]
    ptrs = (ctypes.c_void_p * N)(*[t.ctypes.data for t in Tc])
    nn = (ctypes.c_int64 * N)(*n)
    lib = _lib()
    singular = False
    for r in range(rest):
        col = np.asfortranarray(flat[:, r])
        rc = lib.oracle_sweep(N, nn, ptrs, col.ctypes.data)
        if rc == 2:
            raise RuntimeError("oracle_sweep: bad arguments")
        singular |= rc == 1
        flat[:, r] = col
    if singular:
        raise ZeroDivisionError("a diagonal sum t_{1,i1i1}+...+t_{N,iNiN} is zero")
    return Y


def triangular_sweep_nested(T: Sequence[np.ndarray], C: np.ndarray) -> np.ndarray:
    """Algorithm 1 written as N explicit nested loops (pure Python; tiny inputs).

    Independent of the mixed-radix counter: `itertools.product` over reversed
    ranges with the last mode outermost reproduces the nesting of Algorithm 1.
    """
    N = len(T)
    n = [t.shape[0] for t in T]
    Y = np.array(C, dtype=np.complex128, order="F", copy=True)
    extra = Y.shape[N:]
    for tail in itertools.product(*[range(e) for e in extra]):
        for rev in itertools.product(*[range(nj - 1, -1, -1) for nj in reversed(n)]):
            ii = tuple(reversed(rev))                         # i_N outermost loop
            num = Y[ii + tail]
            den = 0j
            for j in range(N):
                den += T[j][ii[j], ii[j]]
                for k in range(ii[j] + 1, n[j]):
                    kk = ii[:j] + (k,) + ii[j + 1:]
                    num -= T[j][ii[j], k] * Y[kk + tail]
            Y[ii + tail] = num / den
    return Y


# ----------------------------------------------------------------------------
# Drivers
# ----------------------------------------------------------------------------

def solve_with_factors(factors, B: np.ndarray,
                       sweep: Callable = triangular_sweep,
                       timings: Optional[dict] = None) -> np.ndarray:
    """Algorithm 3 with given Schur factors [(U_j or None, T_j)]."""
    U = [f[0] for f in factors]
    T = [f[1] for f in factors]
    t0 = time.perf_counter()
    C = forward_transform(U, B)
    t1 = time.perf_counter()
    Y = sweep(T, C)
    t2 = time.perf_counter()
    X = back_transform(U, Y)
    t3 = time.perf_counter()
    if timings is not None:
        timings["forward"] = timings.get("forward", 0.0) + (t1 - t0)
        timings["sweep"] = timings.get("sweep", 0.0) + (t2 - t1)
        timings["back"] = timings.get("back", 0.0) + (t3 - t2)
    return X


def solve(A: Sequence[np.ndarray], B: np.ndarray, timings: Optional[dict] = None,
          sort=None) -> np.ndarray:
    """X with sum_j A_j (x)_j X = B  (Algorithm 3: Schur, forward, sweep, back)."""
    t0 = time.perf_counter()
    factors = schur_factors(A, sort=sort)
    if timings is not None:
        timings["setup"] = timings.get("setup", 0.0) + (time.perf_counter() - t0)
    return solve_with_factors(factors, B, timings=timings)


# ----------------------------------------------------------------------------
# Theorem 1 (Section 3): the linear ODE X_t = sum_j A_j (x)_j X + B
# ----------------------------------------------------------------------------

def evolve_rhs(A: Sequence[np.ndarray], B: np.ndarray, X0: np.ndarray, t: float) -> np.ndarray:
    """F of Eq. (C): exp(t A_N) (x)_N ( ... exp(t A_1) (x)_1 (sum_j A_j (x)_j X0 + B)) - B.

    The matrix exponentials are scipy's (a library primitive); the mode
    products are applied in the order 1..N written in Eq. (C)."""
    if np.shape(X0) != np.shape(B):
        raise ValueError("X0 and B must have the same shape")
    W = apply_operator(A, X0) + B
    for j, a in enumerate(A):
        W = mode_product(scipy.linalg.expm(t * np.asarray(a, dtype=np.complex128)), W, j)
    return W - B


def evolve(A: Sequence[np.ndarray], B: np.ndarray, X0: np.ndarray, t: float) -> np.ndarray:
    """X(t) of X_t = sum_j A_j (x)_j X + B, X(0) = X0 (Theorem 1): the solution of
    the Sylvester equation sum_j A_j (x)_j X(t) = F, Eq. (sylvesterNDC)-(C), by
    Algorithm 3."""
    return solve(A, evolve_rhs(A, B, X0, t))


def set_threads(k: int) -> None:
    """Threads that the calling thread's mode products spread their independent
    fibres over (1: stay on the calling thread, for callers that run several
    oracle solves at once)."""
    _lib().oracle_set_threads(int(k))


# ----------------------------------------------------------------------------
# Error measures (Section 5 uses the absolute max-norm; relative is its ratio)
# ----------------------------------------------------------------------------

def rel_err(X: np.ndarray, Xref: np.ndarray) -> float:
    """||vec(X) - vec(Xref)||_inf / ||vec(Xref)||_inf."""
    den = float(np.max(np.abs(Xref))) if Xref.size else 0.0
    num = float(np.max(np.abs(X - Xref))) if X.size else 0.0
    return num / den if den > 0 else num


def backward_error(A: Sequence[np.ndarray], X: np.ndarray, B: np.ndarray) -> float:
    """||B - sum_j A_j (x)_j X||_inf / (sum_j ||A_j||_inf ||X||_inf + ||B||_inf)."""
    R = residual(A, X, B)
    anorm = sum(float(np.max(np.sum(np.abs(a), axis=1))) for a in A)
    xn = float(np.max(np.abs(X)))
    bn = float(np.max(np.abs(B)))
    return float(np.max(np.abs(R))) / (anorm * xn + bn)
