"""Pins of the oracle's error measures, which every parity assertion uses.

Section 5 measures the absolute max-norm error ||vec(X) - vec(X_num)||_inf;
the tests use it relative to the reference's max-norm, and bound the backward
error eta = ||B - sum_j A_j (x)_j X||_inf / (sum_j ||A_j||_inf ||X||_inf + ||B||_inf)
where the oracle cannot run.  Here both helpers get hand-computed inputs whose
values are worked out in the comments, and plausible wrong variants (a sum or
Frobenius norm, the other argument's norm as denominator, the largest real or
imaginary part instead of the modulus, the column-sum norm of A_j, a mode
product over A_j's first index) are shown to give other values, so that a
helper rewritten into one of them fails the pinned value."""
import numpy as np
import pytest

import oracle


def _pair():
    # Xref holds 10, 6i, -8 (and zeros) in a 2 x 2 x 2 tensor; X differs by
    # 3 + 4i at the first entry and by 1 at the third: |X - Xref| has max
    # |3 + 4i| = 5, and max |Xref| = 10, so the relative max-norm error is 1/2.
    Xref = np.zeros((2, 2, 2), dtype=np.complex128, order="F")
    Xref[0, 0, 0] = 10.0
    Xref[1, 1, 0] = 6.0j
    Xref[0, 1, 1] = -8.0
    X = Xref.copy(order="F")
    X[0, 0, 0] += 3.0 + 4.0j
    X[0, 1, 1] += 1.0
    return X, Xref


def test_rel_err_hand_computed():
    X, Xref = _pair()
    assert oracle.rel_err(X, Xref) == 0.5
    # argument order matters: the reference's norm is the denominator
    assert oracle.rel_err(Xref, X) == pytest.approx(5.0 / abs(13.0 + 4.0j), rel=1e-15)
    assert oracle.rel_err(Xref, Xref) == 0.0
    # an empty pair and a zero reference (absolute error then)
    assert oracle.rel_err(np.zeros(0), np.zeros(0)) == 0.0
    assert oracle.rel_err(np.array([3.0 + 4.0j]), np.zeros(1)) == 5.0


def test_rel_err_wrong_variants_give_other_values():
    X, Xref = _pair()
    d = (X - Xref).ravel()
    r = Xref.ravel()
    variants = {
        "sum norm": np.abs(d).sum() / np.abs(r).sum(),                    # 6 / 24
        "Frobenius": np.linalg.norm(d) / np.linalg.norm(r),               # sqrt(26 / 200)
        "X as denominator": np.abs(d).max() / np.abs(X).max(),            # 5 / |13 + 4i|
        "largest part": np.abs(d.view(float)).max() / np.abs(r.view(float)).max(),  # 4 / 10
        "mean error": np.abs(d).mean() / np.abs(r).max(),                   # (6 / 8) / 10
        "last axis slice": np.abs(X - Xref)[..., 1].max() / np.abs(Xref)[..., 1].max(),  # 1 / 8
    }
    for name, v in variants.items():
        assert abs(v - 0.5) > 0.05, name


def _problem():
    # N = 2, both modes of size 2:
    #   A_1 = [[1, 2], [0, 1/2]]   row sums 3, 1/2 -> ||A_1||_inf = 3 (column sums 1, 5/2)
    #   A_2 = [[1, 0], [i, 3]]     row sums 1, 4   -> ||A_2||_inf = 4 (column sums 2, 3)
    #   X = 2 e_(1,1):  (A_1 (x)_1 X)_(i1,i2) = sum_k A_1[i1,k] X[k,i2] = 2 A_1[i1,1] [i2 = 1]
    #                   -> [[2, 0], [0, 0]]
    #                   (A_2 (x)_2 X)_(i1,i2) = sum_k A_2[i2,k] X[i1,k] = 2 A_2[i2,1] [i1 = 1]
    #                   -> [[2, 2i], [0, 0]]
    #   B = [[4, 0], [0, 0]]  ->  R = B - [[4, 2i], [0, 0]] = [[0, -2i], [0, 0]], ||R|| = 2
    #   eta = 2 / ((3 + 4) * 2 + 4) = 1/9
    A1 = np.array([[1.0, 2.0], [0.0, 0.5]], dtype=np.complex128)
    A2 = np.array([[1.0, 0.0], [1.0j, 3.0]], dtype=np.complex128)
    X = np.zeros((2, 2), dtype=np.complex128, order="F")
    X[0, 0] = 2.0
    B = np.zeros((2, 2), dtype=np.complex128, order="F")
    B[0, 0] = 4.0
    return [A1, A2], X, B


def test_backward_error_hand_computed():
    A, X, B = _problem()
    R = oracle.residual(A, X, B)
    assert np.array_equal(R, np.array([[0, -2j], [0, 0]]))
    assert oracle.backward_error(A, X, B) == pytest.approx(1.0 / 9.0, rel=1e-15)
    # an exact solution has eta = 0: X = 1 with A_1 = 1 and A_2 = 2 (scalars) and B = 3
    assert oracle.backward_error([np.array([[1.0 + 0j]]), np.array([[2.0 + 0j]])],
                                 np.ones((1, 1), complex), 3.0 * np.ones((1, 1), complex)) == 0.0


def test_backward_error_wrong_variants_give_other_values():
    A, X, B = _problem()
    R = oracle.residual(A, X, B)
    rn, xn, bn = np.abs(R).max(), np.abs(X).max(), np.abs(B).max()
    col = sum(np.abs(a).sum(axis=0).max() for a in A)                    # 2.5 + 3
    fro = sum(np.linalg.norm(a) for a in A)
    # mode products over A_j's first index (transposed operators): R = [[0, 0], [-4, 0]]
    Rt = B - oracle.apply_operator([a.T for a in A], X)
    variants = {
        "column-sum norm": rn / (col * xn + bn),                           # 2 / 15
        "Frobenius norm": rn / (fro * xn + bn),
        "no ||B||": rn / (7.0 * xn),                                        # 1 / 7
        "transposed A_j": np.abs(Rt).max() / (7.0 * xn + bn),              # 4 / 18
    }
    for name, v in variants.items():
        assert abs(v - 1.0 / 9.0) > 0.005, name
