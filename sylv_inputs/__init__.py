"""Seeded synthetic inputs for the N-dimensional Sylvester tensor equation.

    sum_j A_j (x)_j X = B        (the mode-j product contracts A_j's second index
                                  with X's j-th index; Section 1, Eq. (sylvesterND))

This module is shared by the CPU oracle, the CUDA parity tests and the
benchmark.  It holds no arithmetic of the solution method: it only draws
coefficient matrices and right-hand sides from `numpy.random.default_rng`.

Layout conventions (Section 2.2, Eq. (index)): tensors are column-major with
i_1 fastest; complex values are stored interleaved (re, im) as complex128.
A right-hand-side index, when present, is one extra trailing axis.

Recipe (seed 0 unless stated):
  * dense operators  A = (randn(n,n) + 1j*randn(n,n)) / sqrt(n) + shift*I,
    drawn for j = 1..N in order, real block first then imaginary block;
  * singleton modes (n_j = 1) use the scalar A_j = [1.5];
  * B (and any manufactured X) is unit-variance complex Gaussian
    (randn + 1j*randn)/sqrt(2), drawn after every operator, in chunks of
    2**26 entries in memory order, real part then imaginary part per chunk;
  * the batched workload draws its 512 x 3 shapes with
    rng.integers(16, 97, size=(512, 3)) before any matrix;
  * the periodic advection-diffusion operator is 0.01*D2 + 0.5*D1 + I with
    centred differences on x_m = 2*pi*m/n, h = 2*pi/n;
  * real problems (the real-arithmetic variant): A = randn(n,n)/sqrt(n) +
    shift*I drawn mode by mode, singleton modes [1.5], B real unit-variance
    Gaussian drawn after every operator in chunks of 2**26 entries.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

CHUNK = 1 << 26


@dataclass
class Problem:
    """One equation: operators A_j (complex128, n_j x n_j), right-hand side B.

    B has shape (n_1, ..., n_N, nrhs) in Fortran (column-major) order; the
    trailing axis is the right-hand-side index.
    """

    A: List[np.ndarray]
    B: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return tuple(a.shape[0] for a in self.A)

    @property
    def nrhs(self) -> int:
        return int(self.B.shape[-1])

    @property
    def n_tot(self) -> int:
        return int(np.prod(self.shape, dtype=np.int64))


def gaussian_operator(rng: np.random.Generator, n: int, shift: float,
                      scale: Optional[float] = None) -> np.ndarray:
    """(randn + i randn) * scale + shift * I, scale defaulting to 1/sqrt(n)."""
    if scale is None:
        scale = 1.0 / math.sqrt(n)
    re = rng.standard_normal((n, n))
    im = rng.standard_normal((n, n))
    a = (re + 1j * im) * scale
    a[np.diag_indices(n)] += shift
    return a


def complex_gaussian(rng: np.random.Generator, shape: Sequence[int]) -> np.ndarray:
    """Unit-variance complex Gaussian tensor in Fortran order, drawn in chunks."""
    total = int(np.prod(shape, dtype=np.int64))
    out = np.empty(total, dtype=np.complex128)
    view = out.view(np.float64).reshape(total, 2)
    s = 1.0 / math.sqrt(2.0)
    for start in range(0, total, CHUNK):
        stop = min(total, start + CHUNK)
        m = stop - start
        view[start:stop, 0] = rng.standard_normal(m) * s
        view[start:stop, 1] = rng.standard_normal(m) * s
    return out.reshape(tuple(shape), order="F")


def random_problem(shape: Sequence[int], nrhs: int = 1, seed: int = 0,
                   shift: float = 3.0, scale: Optional[float] = None,
                   singleton_value: complex = 1.5, name: str = "") -> Problem:
    """Dense Gaussian operators per mode (scalar `singleton_value` for n_j = 1)."""
    rng = np.random.default_rng(seed)
    A = []
    for n in shape:
        if n == 1:
            A.append(np.array([[complex(singleton_value)]], dtype=np.complex128))
        else:
            A.append(gaussian_operator(rng, int(n), shift, scale))
    B = complex_gaussian(rng, tuple(shape) + (nrhs,))
    return Problem(A=A, B=B, name=name or f"random{tuple(shape)}x{nrhs}")


def real_gaussian(rng: np.random.Generator, shape: Sequence[int]) -> np.ndarray:
    """Unit-variance real Gaussian tensor in Fortran order, drawn in chunks."""
    total = int(np.prod(shape, dtype=np.int64))
    out = np.empty(total, dtype=np.float64)
    for start in range(0, total, CHUNK):
        stop = min(total, start + CHUNK)
        out[start:stop] = rng.standard_normal(stop - start)
    return out.reshape(tuple(shape), order="F")


def random_real_problem(shape: Sequence[int], nrhs: int = 1, seed: int = 0,
                        shift: float = 3.0, scale: Optional[float] = None,
                        singleton_value: float = 1.5, name: str = "") -> Problem:
    """Real dense Gaussian operators randn/sqrt(n) + shift I and a real B."""
    rng = np.random.default_rng(seed)
    A = []
    for n in shape:
        if n == 1:
            A.append(np.array([[float(singleton_value)]]))
        else:
            a = rng.standard_normal((int(n), int(n))) * (
                1.0 / math.sqrt(n) if scale is None else scale)
            a[np.diag_indices(int(n))] += shift
            A.append(a)
    B = real_gaussian(rng, tuple(shape) + (nrhs,))
    return Problem(A=A, B=B, name=name or f"real{tuple(shape)}x{nrhs}")


def real_cube_n64_N4(seed: int = 0) -> Problem:
    """Real N=4, n=64: 16,777,216 entries (134 MB in float64)."""
    return random_real_problem((64,) * 4, 1, seed, shift=3.0, name="real_N4_n64")


def periodic_advdiff_operator(n: int, nu: float = 0.01, c: float = 0.5,
                              mass: float = 1.0) -> np.ndarray:
    """nu*D2 + c*D1 + mass*I with centred periodic differences, h = 2*pi/n.

    (S u)_m = u_{m+1};  D1 = (S - S^-1)/(2h);  D2 = (S - 2I + S^-1)/h^2.
    """
    h = 2.0 * math.pi / n
    S = np.roll(np.eye(n), 1, axis=1)  # S[m, m+1] = 1
    Sinv = S.T
    D1 = (S - Sinv) / (2.0 * h)
    D2 = (S - 2.0 * np.eye(n) + Sinv) / (h * h)
    return (nu * D2 + c * D1 + mass * np.eye(n)).astype(np.complex128)


# --------------------------------------------------------------------------
# The five workloads of the benchmark suite (sizes as named in each function)
# --------------------------------------------------------------------------

def cube_n8_N3(seed: int = 0) -> Problem:
    """N=3, n=8: 512 entries, A = (randn+i randn)/sqrt(8) + 3I."""
    return random_problem((8, 8, 8), 1, seed, shift=3.0, name="N3_n8")


def cube_n64_N4(seed: int = 0) -> Problem:
    """N=4, n=64: 16,777,216 entries (268 MB in complex128)."""
    return random_problem((64,) * 4, 1, seed, shift=3.0, name="N4_n64")


def cube_n19_N7(seed: int = 0) -> Problem:
    """N=7, n=19: 893,871,739 entries (14.3 GB in complex128)."""
    return random_problem((19,) * 7, 1, seed, shift=3.0, name="N7_n19")


def binary_N29_shape():
    """n_j = 2 except modes 5 and 17 (1-based), which are singletons."""
    return tuple(1 if j in (5, 17) else 2 for j in range(1, 30))


def binary_N29(seed: int = 0) -> Problem:
    """N=29 with 2x2 operators (randn+i randn)/sqrt(2) + 2I and two [1.5] singletons."""
    return random_problem(binary_N29_shape(), 1, seed, shift=2.0, name="N29_n2")


def batch_shapes(count: int = 512, seed: int = 0, lo: int = 16, hi: int = 96):
    rng = np.random.default_rng(seed)
    return rng, [tuple(int(v) for v in row) for row in rng.integers(lo, hi + 1, size=(count, 3))]


def uneven_batch(count: int = 512, nrhs: int = 4, seed: int = 0, lo: int = 16,
                 hi: int = 96) -> List[Problem]:
    """`count` independent N=3 equations, n_k ~ U{lo..hi}, nrhs right-hand sides each."""
    rng, shapes = batch_shapes(count, seed, lo, hi)
    out = []
    for e, shp in enumerate(shapes):
        A = [gaussian_operator(rng, n, 3.0) for n in shp]
        out.append(Problem(A=A, B=None, name=f"batch{e}", meta={"shape": shp}))
    for p in out:
        p.B = complex_gaussian(rng, p.meta["shape"] + (nrhs,))
    return out


def advdiff_n48(nrhs: int = 32, seed: int = 0, n: int = 48) -> Problem:
    """N=3, n=48 periodic advection-diffusion operator in every mode, 32 RHS."""
    rng = np.random.default_rng(seed)
    A = [periodic_advdiff_operator(n) for _ in range(3)]
    B = complex_gaussian(rng, (n, n, n, nrhs))
    return Problem(A=A, B=B, name="advdiff_n48")


def manufactured(shape: Sequence[int], nrhs: int = 1, seed: int = 0,
                 shift: float = 3.0, scale: Optional[float] = None):
    """Operators plus a drawn solution X (the caller forms B from X)."""
    p = random_problem(shape, nrhs, seed, shift=shift, scale=scale)
    rng = np.random.default_rng(seed + 7919)
    X = complex_gaussian(rng, tuple(shape) + (nrhs,))
    return p.A, X


def initial_state(shape: Sequence[int], nrhs: int = 1, seed: int = 1) -> np.ndarray:
    """Initial value X(0) for the ODE X_t = sum_j A_j (x)_j X + B (Theorem 1):
    a unit-variance complex Gaussian tensor from its own seeded stream, with
    the trailing right-hand-side axis of Problem.B."""
    return complex_gaussian(np.random.default_rng(seed), tuple(shape) + (nrhs,))
