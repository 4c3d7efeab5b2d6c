"""Pins for the CPU oracle (no GPU).  Each test checks the oracle against
something other than itself: the paper's worked example, a dense solve of the
Kronecker-sum system, textbook solvers, closed forms, invariants and planted
mistakes."""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
import oracle.bartels_stewart as bs
import sylv_inputs as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers --

def kron_sum_matrix(A):
    """A_N (+) ... (+) A_1 = sum_j I (x) ... (x) A_j (x) ... (x) I (Eq. (systvec)).

    Kronecker factors run from mode N (leftmost) down to mode 1, matching the
    column-major vec of Section 1."""
    n = [a.shape[0] for a in A]
    N = len(A)
    K = 0
    for j in range(N):
        f = None
        for m in reversed(range(N)):
            blk = A[m] if m == j else np.eye(n[m])
            f = blk if f is None else np.kron(f, blk)
        K = K + f
    return K


def brute_force(A, B):
    """Dense LU solve of the Kronecker-sum system, one right-hand side per column."""
    n = [a.shape[0] for a in A]
    lead = int(np.prod(n))
    K = kron_sum_matrix(A)
    Bm = np.asarray(B).reshape(lead, -1, order="F")
    X = np.linalg.solve(K, Bm)
    return X.reshape(B.shape, order="F")


def rand_ops(shape, seed, shift=3.0):
    p = si.random_problem(shape, nrhs=2, seed=seed, shift=shift)
    return p.A, p.B


SHAPES = [(3,), (4, 1), (2, 3), (3, 2, 4), (2, 1, 3), (1, 4), (2, 2, 2, 2),
          (3, 1, 1, 2), (1, 1, 3), (5, 2, 3), (2, 3, 2, 2, 1)]


# ------------------------------------------------------------- index pins --

def test_index_worked_example_golden():
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLDEN, "index_example.txt"))
            if l.strip() and not l.startswith("#")]
    n = (5, 2, 3)
    order = oracle.counter_order(n)
    assert len(order) == 30 and len(set(order)) == 30
    for pos, i1, i2, i3, idx in rows:
        assert oracle.linear_index((i1, i2, i3), n) == idx
        assert order[pos - 1] == (i1, i2, i3)
    # the counter visits linear indices n_tot, n_tot-1, ..., 1 in that order
    assert [oracle.linear_index(t, n) for t in order] == list(range(30, 0, -1))


def test_linear_index_matches_fortran_layout():
    n = (3, 4, 2, 5)
    a = np.arange(np.prod(n)).reshape(n, order="F")
    for ii in itertools.product(*[range(1, v + 1) for v in n]):
        assert a[tuple(i - 1 for i in ii)] == oracle.linear_index(ii, n) - 1


# ----------------------------------------------------- whole-method pins --

@pytest.mark.parametrize("shape", SHAPES)
def test_solve_matches_kronecker_bruteforce(shape):
    A, B = rand_ops(shape, seed=len(shape) * 10 + sum(shape))
    X = oracle.solve(A, B)
    Xb = brute_force(A, B)
    assert oracle.rel_err(X, Xb) < 1e-12


def test_cube_n8_N3_bruteforce_512():
    p = si.cube_n8_N3()
    X = oracle.solve(p.A, p.B)
    Xb = brute_force(p.A, p.B)
    assert oracle.rel_err(X, Xb) < 1e-13


@pytest.mark.parametrize("seed", [0, 1])
def test_two_dimensional_matches_scipy(seed):
    # Eq. (sylvester): A1 X + X A2^T = B  (plain transpose)
    A, B = rand_ops((7, 5), seed)
    X = oracle.solve(A, B[..., 0])
    Xs = scipy.linalg.solve_sylvester(A[0], A[1].T, B[..., 0])
    assert oracle.rel_err(X, Xs) < 1e-12


def test_one_dimensional_is_linear_solve():
    A, B = rand_ops((9,), 3)
    X = oracle.solve(A, B)
    assert oracle.rel_err(X, np.linalg.solve(A[0], B)) < 1e-13


def test_diagonal_closed_form():
    # Remark 1: normal (here diagonal) A_j give y = c / sum_j lambda_{j,i_j}
    rng = np.random.default_rng(5)
    n = (4, 3, 5)
    lam = [rng.standard_normal(v) + 1j * rng.standard_normal(v) + 4 for v in n]
    A = [np.diag(l) for l in lam]
    B = si.complex_gaussian(rng, n)
    den = lam[0][:, None, None] + lam[1][None, :, None] + lam[2][None, None, :]
    assert oracle.rel_err(oracle.solve(A, B), B / den) < 1e-14


def test_circulant_fft_closed_form_advdiff_n48_full_size():
    """The periodic advection-diffusion workload at its full size (48^3, 32 RHS):
    circulant operators are diagonalised by the DFT, so X = IFFT(FFT(B)/Lambda)."""
    p = si.advdiff_n48()
    n = 48
    h = 2 * math.pi / n
    w = 2 * math.pi * np.arange(n) / n
    # (S u)_m = u_{m+1}  ->  DFT eigenvalue e^{i w}
    lam = 0.01 * (2 * np.cos(w) - 2) / h ** 2 + 0.5 * (1j * np.sin(w)) / h + 1.0
    Lam = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    Xf = np.fft.ifftn(np.fft.fftn(p.B, axes=(0, 1, 2)) / Lam[..., None], axes=(0, 1, 2))
    X = oracle.solve(p.A, p.B)
    assert oracle.rel_err(X, Xf) < 1e-12


def test_singleton_reduction():
    # a singleton mode A_j = [a] contributes a to every denominator: the problem
    # equals the one without that mode and with A_1 + a I (Section 4)
    A, B = rand_ops((4, 1, 3, 1), 11)
    a = A[1][0, 0] + A[3][0, 0]
    X = oracle.solve(A, B)
    A_red = [A[0] + a * np.eye(4), A[2]]
    X_red = oracle.solve(A_red, B.reshape(4, 3, 2, order="F"))
    assert oracle.rel_err(X.reshape(4, 3, 2, order="F"), X_red) < 1e-13


def test_manufactured_solution_and_residual_invariant():
    # the paper's own test pattern (Section 5): draw X, form B, solve
    shape = (9, 7, 6, 5)
    A, Xt = si.manufactured(shape, nrhs=2, seed=3)
    B = np.zeros_like(Xt, order="F")
    for j in range(len(A)):            # einsum written independently of the oracle
        letters = "abcd"
        spec = f"z{letters[j]},{letters}r->{letters[:j]}z{letters[j+1:]}r"
        B += np.einsum(spec, A[j], Xt)
    X = oracle.solve(A, B)
    assert oracle.rel_err(X, Xt) < 1e-12
    assert oracle.backward_error(A, X, B) < 1e-15 * 50


def test_schur_ordering_independence():
    A, B = rand_ops((6, 5, 4), 8)
    X1 = oracle.solve(A, B)
    X2 = oracle.solve(A, B, sort="lhp")
    X3 = oracle.solve(A, B, sort="rhp")
    assert oracle.rel_err(X1, X2) < 1e-13 and oracle.rel_err(X1, X3) < 1e-13


def test_mode_permutation_equivariance():
    A, B = rand_ops((5, 3, 4), 9)
    X = oracle.solve(A, B)
    perm = (2, 0, 1)
    Ap = [A[p] for p in perm]
    Bp = np.asfortranarray(np.transpose(B, perm + (3,)))
    Xp = oracle.solve(Ap, Bp)
    assert oracle.rel_err(Xp, np.transpose(X, perm + (3,))) < 1e-13


def test_linearity_in_B():
    A, B = rand_ops((4, 5, 3), 12)
    B2 = si.complex_gaussian(np.random.default_rng(1), B.shape)
    X1, X2 = oracle.solve(A, B), oracle.solve(A, B2)
    X12 = oracle.solve(A, 2.0 * B - 1j * B2)
    assert oracle.rel_err(X12, 2.0 * X1 - 1j * X2) < 1e-13


# --------------------------------------------------------- per-phase pins --

@pytest.mark.parametrize("shape", [(3, 4), (2, 3, 4), (3, 1, 2, 2), (4,)])
def test_sweep_matches_nested_loops_and_triangular_system(shape):
    A, B = rand_ops(shape, 21)
    f = oracle.schur_factors(A)
    T = [t for _, t in f]
    Y = oracle.triangular_sweep(T, B)
    Yn = oracle.triangular_sweep_nested(T, B)     # Algorithm 1 (nested loops)
    assert oracle.rel_err(Y, Yn) < 1e-14
    # sum_j T_j (x)_j Y = C, checked with a dense Kronecker-sum product
    K = kron_sum_matrix(T)
    lead = int(np.prod(shape))
    assert np.allclose(K @ Y.reshape(lead, -1, order="F"), B.reshape(lead, -1, order="F"),
                       rtol=0, atol=1e-12)
    assert np.allclose(np.tril(K, -1), 0)          # Eq. (yi1i2iN) structure


def test_transforms_are_unitary_and_inverse():
    A, B = rand_ops((5, 4, 6), 4)
    U = [u for u, _ in oracle.schur_factors(A)]
    C = oracle.forward_transform(U, B)
    assert abs(np.linalg.norm(C) - np.linalg.norm(B)) < 1e-12 * np.linalg.norm(B)
    assert oracle.rel_err(oracle.back_transform(U, C), B) < 1e-14
    # forward equals the Kronecker form (U_3 (x) U_2 (x) U_1)^* vec(B)
    Kf = np.kron(U[2], np.kron(U[1], U[0])).conj().T
    lead = 120
    assert np.allclose(C.reshape(lead, -1, order="F"), Kf @ B.reshape(lead, -1, order="F"),
                       atol=1e-13)


def test_mode_product_definition_elementwise():
    rng = np.random.default_rng(2)
    X = si.complex_gaussian(rng, (3, 4, 2))
    M = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    Y = oracle.mode_product(M, X, 1)
    for a, i, c in itertools.product(range(3), range(4), range(2)):
        assert abs(Y[a, i, c] - sum(M[i, k] * X[a, k, c] for k in range(4))) < 1e-13


# -------------------------------------------------- planted mistakes ------

def _mut_sweep(kind):
    def sweep(T, C):
        N = len(T)
        n = [t.shape[0] for t in T]
        Y = np.array(C, dtype=np.complex128, order="F", copy=True)
        for tail in itertools.product(*[range(e) for e in Y.shape[N:]]):
            for rev in itertools.product(*[range(v - 1, -1, -1) for v in reversed(n)]):
                ii = tuple(reversed(rev))
                num, den = Y[ii + tail], 0j
                for j in range(N):
                    if not (kind == "drop_mode_den" and j == N - 1):
                        den += T[j][ii[j], ii[j]]
                    hi = n[j] - 1 if kind == "drop_last_k" else n[j]
                    for k in range(ii[j] + 1, hi):
                        kk = ii[:j] + (k,) + ii[j + 1:]
                        t = T[j][k, ii[j]] if kind == "transposed_T" else T[j][ii[j], k]
                        if kind == "wrong_sign":
                            num += t * Y[kk + tail]
                        else:
                            num -= t * Y[kk + tail]
                Y[ii + tail] = num / den
        return Y
    return sweep


@pytest.mark.parametrize("kind", ["wrong_sign", "drop_last_k", "transposed_T", "drop_mode_den"])
def test_planted_sweep_mistakes_are_caught(kind):
    A, B = rand_ops((3, 3, 2), 30)
    f = oracle.schur_factors(A)
    good = oracle.solve_with_factors(f, B, sweep=oracle.triangular_sweep_nested)
    bad = oracle.solve_with_factors(f, B, sweep=_mut_sweep(kind))
    Xb = brute_force(A, B)
    assert oracle.rel_err(good, Xb) < 1e-12
    assert oracle.rel_err(bad, Xb) > 1e-6


@pytest.mark.parametrize("kind", ["contract_first_index", "forward_no_conj", "back_conj"])
def test_planted_transform_mistakes_are_caught(kind, monkeypatch):
    A, B = rand_ops((3, 4, 2), 31)
    Xb = brute_force(A, B)
    if kind == "contract_first_index":
        def mp(M, X, j):
            out = np.tensordot(M, X, axes=([0], [j]))
            return np.asfortranarray(np.moveaxis(out, 0, j))
        monkeypatch.setattr(bs, "mode_product", mp)
    elif kind == "forward_no_conj":
        def fwd(U, B):
            C = np.array(B, order="F", copy=True)
            for j, u in enumerate(U):
                if u is not None:
                    C = bs.mode_product(u.T, C, j)
            return C
        monkeypatch.setattr(bs, "forward_transform", fwd)
    else:
        def back(U, Y):
            X = np.array(Y, order="F", copy=True)
            for j, u in enumerate(U):
                if u is not None:
                    X = bs.mode_product(u.conj(), X, j)
            return X
        monkeypatch.setattr(bs, "back_transform", back)
    bad = bs.solve(A, B)
    assert oracle.rel_err(bad, Xb) > 1e-6


def test_zero_denominator_is_reported():
    # eigenvalue sums that vanish: A_1 = diag(1, 2), A_2 = diag(-1, 5)
    A = [np.diag([1.0 + 0j, 2.0]), np.diag([-1.0 + 0j, 5.0])]
    with pytest.raises(ZeroDivisionError):
        oracle.solve(A, np.ones((2, 2), dtype=np.complex128, order="F"))


def test_stored_cube_n8_solution_matches_bruteforce():
    """The stored oracle solution (tests/golden/make_golden.py) against the dense
    Kronecker solve, so GPU tests can use it without rerunning the oracle."""
    p = si.cube_n8_N3()
    rows = np.loadtxt(os.path.join(GOLDEN, "cube_n8_N3_X.txt"))
    X = (rows[:, 0] + 1j * rows[:, 1]).reshape(p.B.shape, order="F")
    assert oracle.rel_err(X, brute_force(p.A, p.B)) < 1e-13
