"""Pins of the oracle's real-arithmetic variant (real Schur factors,
quasi-triangular sweep with the 2 x 2 diagonal blocks solved together)."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import real_variant as rv
import sylv_inputs as si

from test_oracle import brute_force, kron_sum_matrix

SHAPES = [(3,), (4, 1), (2, 3), (3, 2, 4), (2, 1, 3), (5, 4), (2, 2, 2, 2), (3, 1, 1, 2),
          (6, 5, 3), (2, 3, 2, 2, 1)]


def _has_pairs(factors):
    return any(any(s == 2 for _, s in rv.diagonal_blocks(T)) for Q, T in factors if Q is not None)


@pytest.mark.parametrize("shape", SHAPES)
def test_real_solve_matches_kronecker_bruteforce(shape):
    p = si.random_real_problem(shape, nrhs=2, seed=sum(shape) + len(shape), shift=0.5)
    X = rv.solve_real(p.A, p.B)
    assert X.dtype == np.float64
    assert oracle.rel_err(X, brute_force(p.A, p.B)) < 1e-12


def test_operators_have_complex_pairs():
    # the shift-0.5 draws above produce 2 x 2 blocks (otherwise nothing is pinned)
    count = 0
    for shape in SHAPES:
        p = si.random_real_problem(shape, nrhs=2, seed=sum(shape) + len(shape), shift=0.5)
        count += _has_pairs(rv.real_schur_factors(p.A))
    assert count >= 6


@pytest.mark.parametrize("shape", [(4, 3), (2, 2, 3), (5, 2, 2)])
def test_quasi_triangular_sweep_matches_dense_solve(shape):
    p = si.random_real_problem(shape, nrhs=1, seed=7 + sum(shape), shift=0.5)
    F = rv.real_schur_factors(p.A)
    T = [f[1] for f in F]
    C = p.B
    Y = rv.quasi_triangular_sweep(T, C)
    lead = int(np.prod(shape))
    ref = np.linalg.solve(kron_sum_matrix(T), C.reshape(lead, -1, order="F"))
    assert oracle.rel_err(Y, ref.reshape(C.shape, order="F")) < 1e-12


@pytest.mark.parametrize("seed", range(3))
def test_real_two_dimensional_matches_scipy(seed):
    p = si.random_real_problem((7, 5), nrhs=1, seed=seed, shift=0.3)
    X = rv.solve_real(p.A, p.B)
    ref = scipy.linalg.solve_sylvester(p.A[0], p.A[1].T, p.B[:, :, 0])
    assert oracle.rel_err(X[:, :, 0], ref) < 1e-12


def test_real_solution_equals_complex_solution():
    p = si.random_real_problem((6, 5, 4), nrhs=2, seed=3, shift=1.0)
    Xr = rv.solve_real(p.A, p.B)
    Xc = oracle.solve([a.astype(np.complex128) for a in p.A], p.B.astype(np.complex128))
    assert np.abs(Xc.imag).max() < 1e-12 * np.abs(Xc).max()
    assert oracle.rel_err(Xr, Xc.real) < 1e-12


def test_real_transforms_are_orthogonal_and_inverse():
    p = si.random_real_problem((5, 4, 3), nrhs=1, seed=9)
    Q = [f[0] for f in rv.real_schur_factors(p.A)]
    C = rv.forward_transform_real(Q, p.B)
    assert abs(np.linalg.norm(C) - np.linalg.norm(p.B)) < 1e-12 * np.linalg.norm(p.B)
    assert oracle.rel_err(rv.back_transform_real(Q, C), p.B) < 1e-14


def test_planted_mistake_dropping_the_block_coupling_fails():
    # treating T_j as triangular (the 2 x 2 blocks' subdiagonal ignored) is wrong
    p = si.random_real_problem((4, 3), nrhs=1, seed=5, shift=0.5)
    F = rv.real_schur_factors(p.A)
    assert _has_pairs(F)
    bad = [(Q, np.triu(T)) for Q, T in F]
    X = rv.solve_real_with_factors(bad, p.B)
    assert oracle.rel_err(X, brute_force(p.A, p.B)) > 1e-3


def test_planted_mistake_transposed_factor_fails():
    p = si.random_real_problem((4, 3), nrhs=1, seed=6, shift=0.5)
    F = rv.real_schur_factors(p.A)
    bad = [(None if Q is None else Q.T, T) for Q, T in F]
    X = rv.solve_real_with_factors(bad, p.B)
    assert oracle.rel_err(X, brute_force(p.A, p.B)) > 1e-3
