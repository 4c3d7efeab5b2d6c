"""CPU model of the arithmetic of the tensor-core residual (SYLV_MIXED_FP32_EMU):
base-256 digit splitting of X / 2^eX and A / 2^eA, exact integer digit-pair
products grouped by order t + u (orders 0, 1, 2 exact, orders 5, 4, 3 folded
with FP32 rounding after each 2^-8 Horner step), complex recombination.  The
model checks the error bound the design relies on, independently of the
kernel (which the GPU tests compare with the oracle)."""
import math

import numpy as np
import pytest


def _digits(v, e):
    F = np.floor(np.abs(v) * 2.0 ** (48 - e)).astype(np.uint64)
    s = np.sign(v)
    return [s * ((F >> np.uint64(40 - 8 * t)) & np.uint64(255)).astype(np.float64)
            for t in range(6)]


def _scale(v):
    m = max(np.abs(v.real).max(), np.abs(v.imag).max())
    return math.frexp(float(m))[1] + 1 if m > 0 else 0        # |v| < 2^(e - 1)


def model_product(A, X):
    """[A (x) X] for rows l of X: sum_k A[i, k] X[l, k], as the kernel computes it."""
    n = A.shape[0]
    eX, eA = _scale(X), _scale(A)
    xr, xi = _digits(X.real, eX), _digits(X.imag, eX)
    ar, ai = _digits(A.real, eA), _digits(A.imag, eA)
    f32 = np.float32

    def level(xd, ad, d):                           # orders 0..2: exact integer sums
        out = sum(xd[t] @ ad[d - t].T for t in range(d + 1))
        assert np.abs(out).max() < 2 ** 24          # exact in the FP32 accumulator
        return out

    def folded(xd, ad):                             # orders 5, 4, 3 with FP32 rounding
        S = np.zeros((X.shape[0], n), dtype=f32)
        for d in (5, 4, 3):
            S = (S * f32(2.0 ** -8)).astype(f32)
            for t in range(d + 1):
                S = (S + (xd[t] @ ad[d - t].T).astype(f32)).astype(f32)
        return S.astype(np.float64)

    acc = [tuple(level(xd, ad, d) for xd, ad in ((xr, ar), (xr, ai), (xi, ar), (xi, ai)))
           for d in range(3)]
    acc.append(tuple(folded(xd, ad) for xd, ad in ((xr, ar), (xr, ai), (xi, ar), (xi, ai))))
    re = sum(2.0 ** (-8 * d) * (acc[d][0] - acc[d][3]) for d in range(4))
    im = sum(2.0 ** (-8 * d) * (acc[d][2] + acc[d][1]) for d in range(4))
    return (re + 1j * im) * 2.0 ** (eX + eA - 16)


@pytest.mark.parametrize("n", [8, 16, 40, 64])
@pytest.mark.parametrize("spread", [0.0, 6.0])
def test_digit_products_meet_the_error_bound(n, spread):
    rng = np.random.default_rng(n + int(spread))
    A = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n) \
        + 3 * np.eye(n)
    X = rng.standard_normal((64, n)) + 1j * rng.standard_normal((64, n))
    X *= 10.0 ** (spread * (rng.random((64, 1)) - 0.5))     # rows over `spread` decades
    exact = X @ A.T
    err = np.abs(model_product(A, X) - exact).max()
    bound = 2.0 ** -43 * n * np.abs(A).max() * np.abs(X).max()
    assert err < bound


def test_dropping_order_three_breaks_the_bound():
    # planted mistake: without the folded accumulator (orders >= 3) the error is
    # ~2^-26, far above the bound; the bound is therefore not vacuous
    rng = np.random.default_rng(1)
    n = 64
    A = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / 8 + 3 * np.eye(n)
    X = rng.standard_normal((64, n)) + 1j * rng.standard_normal((64, n))
    eX, eA = _scale(X), _scale(A)
    xr, xi = _digits(X.real, eX), _digits(X.imag, eX)
    ar, ai = _digits(A.real, eA), _digits(A.imag, eA)
    re = sum(2.0 ** (-8 * d) * sum(xr[t] @ ar[d - t].T - xi[t] @ ai[d - t].T
                                    for t in range(d + 1)) for d in range(3))
    approx = re * 2.0 ** (eX + eA - 16)
    err = np.abs(approx - (X @ A.T).real).max()
    assert err > 2.0 ** -43 * n * np.abs(A).max() * np.abs(X).max() * 100
