"""Pins for the oracle's ODE solution (Theorem 1, Section 3): X(t) for
X_t = sum_j A_j (x)_j X + B, X(0) = X0.  Each test checks it against something
other than the theorem's own formula: the exponential of the augmented
Kronecker-sum matrix, the scalar closed form, a Runge-Kutta integration (the
experiment of Section 5.2), and the t = 0 / steady-state limits."""
import numpy as np
import pytest
import scipy.linalg

import oracle
import oracle.bartels_stewart as bs

from test_oracle import kron_sum_matrix


def _ops(shape, seed, shift=0.0):
    rng = np.random.default_rng(seed)
    A = []
    for n in shape:
        a = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
        A.append(a + shift * np.eye(n) if n > 1 else np.array([[1.5 + 0.25j]]))
    return A, rng


def _tensor(rng, shape):
    return np.asfortranarray((rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
                             / np.sqrt(2))


def _augmented(A, B, X0, t):
    """[y(t); 1] = expm(t [[K, c], [0, 0]]) [y0; 1] for y' = K y + c (vec form,
    Eq. (systvec)), one right-hand side per trailing column."""
    n = [a.shape[0] for a in A]
    lead = int(np.prod(n))
    K = kron_sum_matrix(A)
    Bm = np.asarray(B).reshape(lead, -1, order="F")
    Xm = np.asarray(X0).reshape(lead, -1, order="F")
    out = np.empty_like(Xm)
    for c in range(Bm.shape[1]):
        M = np.zeros((lead + 1, lead + 1), dtype=np.complex128)
        M[:lead, :lead] = K
        M[:lead, lead] = Bm[:, c]
        v = scipy.linalg.expm(t * M) @ np.concatenate([Xm[:, c], [1.0]])
        out[:, c] = v[:lead]
    return out.reshape(X0.shape, order="F")


SHAPES = [(3,), (2, 3), (3, 1, 2), (2, 2, 2), (4, 3), (2, 1, 3, 2)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("t", [0.37, 1.3])
def test_evolve_matches_augmented_exponential(shape, t):
    A, rng = _ops(shape, 1 + len(shape), shift=0.5)
    full = shape + (2,)
    B, X0 = _tensor(rng, full), _tensor(rng, full)
    X = oracle.evolve(A, B, X0, t)
    assert oracle.rel_err(X, _augmented(A, B, X0, t)) < 1e-12


def test_evolve_diagonal_closed_form():
    rng = np.random.default_rng(5)
    shape = (4, 3, 5)
    lam = [rng.standard_normal(n) + 1j * rng.standard_normal(n) + 1.0 for n in shape]
    A = [np.diag(l) for l in lam]
    B, X0 = _tensor(rng, shape), _tensor(rng, shape)
    t = 0.8
    L = lam[0][:, None, None] + lam[1][None, :, None] + lam[2][None, None, :]
    E = np.exp(t * L)
    exact = E * X0 + (E - 1.0) / L * B
    assert oracle.rel_err(oracle.evolve(A, B, X0, t), exact) < 1e-13


def test_evolve_runge_kutta_seven_modes():
    # the experiment of Section 5.2: N = 7, 2 x 3 x ... x 8, t = 0.1, RK4
    shape = (2, 3, 4, 5, 6, 7, 8)
    A, rng = _ops(shape, 7)
    B, X0 = _tensor(rng, shape), _tensor(rng, shape)
    t = 0.1
    X = oracle.evolve(A, B, X0, t)

    def rk4(steps):
        f = lambda Z: oracle.apply_operator(A, Z) + B
        dt = t / steps
        Z = X0.copy()
        for _ in range(steps):
            k1 = f(Z)
            k2 = f(Z + dt / 2 * k1)
            k3 = f(Z + dt / 2 * k2)
            k4 = f(Z + dt * k3)
            Z = Z + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        return Z

    e50, e100 = oracle.rel_err(rk4(50), X), oracle.rel_err(rk4(100), X)
    assert e100 < 2e-11
    assert 10.0 < e50 / e100 < 22.0          # fourth-order convergence towards X(t)


def test_evolve_time_zero_and_steady_state():
    A, rng = _ops((3, 4, 2), 9, shift=2.0)
    B, X0 = _tensor(rng, (3, 4, 2)), _tensor(rng, (3, 4, 2))
    assert oracle.rel_err(oracle.evolve(A, B, X0, 0.0), X0) < 1e-13
    Xs = oracle.solve(A, -B)                 # sum_j A_j (x)_j Xs + B = 0
    assert oracle.rel_err(oracle.evolve(A, B, Xs, 0.6), Xs) < 1e-12


@pytest.mark.parametrize("kind", ["transposed_exponential", "missing_minus_B", "no_forcing"])
def test_planted_evolve_mistakes_are_caught(kind, monkeypatch):
    A, rng = _ops((3, 2, 3), 11, shift=0.5)
    B, X0 = _tensor(rng, (3, 2, 3)), _tensor(rng, (3, 2, 3))
    ref = _augmented(A, B, X0, 0.7)

    def bad_rhs(A_, B_, X0_, t_):
        W = bs.apply_operator(A_, X0_) + (0 if kind == "no_forcing" else B_)
        for j, a in enumerate(A_):
            E = scipy.linalg.expm(t_ * a)
            W = bs.mode_product(E.T if kind == "transposed_exponential" else E, W, j)
        return W if kind == "missing_minus_B" else W - B_

    monkeypatch.setattr(bs, "evolve_rhs", bad_rhs)
    assert oracle.rel_err(bs.evolve(A, B, X0, 0.7), ref) > 1e-6
