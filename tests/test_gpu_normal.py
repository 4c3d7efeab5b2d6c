"""Normal operators (Section 2, Remark 1): the plan detects Schur factors that
are diagonal to rounding and runs the sweep as the entrywise division of
Eq. (yi1i2iNdiag).  Results are compared with the oracle, which always runs
the full triangular sweep of Algorithm 3."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import sylv_inputs as si
from paper_2412_15840_gb300 import Plan, from_device, to_device
from paper_2412_15840_gb300.build import build

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def built():
    build()
    assert torch.cuda.is_available()


def _hermitian(n, rng, shift):
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return (M + M.conj().T) / np.sqrt(8 * n) + shift * np.eye(n)


def _unitary_normal(n, rng, shift):
    # U diag(lambda) U^*: normal, not Hermitian
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    lam = rng.standard_normal(n) + 1j * rng.standard_normal(n) + shift
    return (Q * lam) @ Q.conj().T


def _rhs(shape, nrhs, seed):
    rng = np.random.default_rng(seed)
    full = tuple(shape) + (nrhs,)
    return (rng.standard_normal(full) + 1j * rng.standard_normal(full)) / np.sqrt(2)


def _solve(A, B, prec, **kw):
    plan = Plan(A=A, nrhs=B.shape[-1], prec=prec, **kw)
    X, info = plan.solve(to_device(B), info=True)
    return from_device(X, B.shape), info


def _check(A, B, prec, expect_diag=True):
    X, info = _solve(A, B, prec)
    assert info["status"] == 0
    assert info["diagonal_sweep"] == expect_diag
    Xo = oracle.solve(A, B)
    assert oracle.rel_err(X, Xo) < TOL[prec]
    return X


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_circulant_advection_diffusion(prec):
    A1 = si.periodic_advdiff_operator(16)
    _check([A1, A1, A1], _rhs((16, 16, 16), 4, 1), prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_exactly_diagonal_with_singleton(prec):
    rng = np.random.default_rng(2)
    A = [np.diag(rng.standard_normal(n) + 1j * rng.standard_normal(n) + 3) for n in (7, 1, 5, 9)]
    A[1] = np.array([[1.5]])
    _check(A, _rhs((7, 1, 5, 9), 2, 3), prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_hermitian_and_unitary_normal(prec):
    rng = np.random.default_rng(4)
    A = [_hermitian(12, rng, 3.0), _unitary_normal(10, rng, 3.0), _hermitian(8, rng, 2.0)]
    _check(A, _rhs((12, 10, 8), 3, 5), prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_many_modes_of_size_two(prec):
    # 14 modes: the head table covers 12 of them (4096 entries), two are decoded per column
    rng = np.random.default_rng(6)
    A = [_hermitian(2, rng, 2.0) for _ in range(14)]
    A[4] = np.array([[1.5]])
    shape = tuple(a.shape[0] for a in A)
    _check(A, _rhs(shape, 1, 7), prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_head_columns_cross_chunks(prec):
    # head product 600 does not divide the 2048-entry chunks: columns straddle them
    rng = np.random.default_rng(8)
    A = [_unitary_normal(600, rng, 3.0), _hermitian(9, rng, 1.0)]
    _check(A, _rhs((600, 9), 2, 9), prec)


def test_general_sweep_forced_matches():
    A1 = si.periodic_advdiff_operator(12)
    A = [A1, A1, A1]
    B = _rhs((12, 12, 12), 2, 10)
    Xd, infd = _solve(A, B, "fp64")
    Xg, infg = _solve(A, B, "fp64", general_sweep=True)
    assert infd["diagonal_sweep"] and not infg["diagonal_sweep"]
    assert oracle.rel_err(Xd, Xg) < 1e-13


def test_non_normal_takes_the_triangular_sweep():
    p = si.random_problem((10, 9, 8), 1, seed=11)
    _check(p.A, p.B, "fp64", expect_diag=False)
    # a normal operator plus a small non-normal part is still non-normal
    rng = np.random.default_rng(12)
    A = [_hermitian(10, rng, 3.0) for _ in range(3)]
    A[1] = A[1] + 1e-9 * np.triu(rng.standard_normal((10, 10)), 1)
    _check(A, _rhs((10, 10, 10), 1, 13), "fp64", expect_diag=False)


def test_autotune_with_diagonal_sweep():
    A1 = si.periodic_advdiff_operator(16)
    plan = Plan(A=[A1, A1], nrhs=3, prec="mixed")
    block, ms = plan.autotune()
    assert ms > 0
    B = _rhs((16, 16), 3, 14)
    X = from_device(plan.solve(to_device(B)), B.shape)
    assert oracle.rel_err(X, oracle.solve([A1, A1], B)) < 1e-10
