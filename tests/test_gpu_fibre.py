"""The FP32 transform pass that gives one thread a whole fibre (modes with
n <= 24 outside the TMA-fed tensor-core pass), through the C ABI.

Mixed-precision solves against the FP64 CPU oracle (relative max-norm error
1e-10 after refinement) on shapes that send every register block of the pass
(n up to 8, 12, 16, 20, 24) through it: the first mode (contiguous fibres,
L = 1), odd L, a fused CUDA-core group before it, a last grid-stride round that
is ragged, several right-hand sides.  A mixed solve runs every epilogue of the
pass: the first forward pass reads complex128 B, the middle passes complex64,
the last back pass writes complex128 X with its norm, and the refinement's
back transform adds the correction into X."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import sylv_inputs as si
from paper_2412_15840_gb300 import Plan, from_device, to_device
from paper_2412_15840_gb300.build import build

pytestmark = pytest.mark.gpu

TOL = 1e-10

# shape, right-hand sides, fibre passes the plan must choose
CASES = [
    ((23, 9, 17), 2, 3),        # every mode: L = 1, L = 23 (n = 9), L = 207
    ((5, 13, 21, 3), 1, 2),     # (5, 13) fused on the CUDA cores, then n = 21 and n = 3
    ((24, 24, 7), 3, 3),        # n = 24 at L = 1 and L = 24, n = 7 at L = 576
    ((12, 11, 10, 9), 1, 1),    # (12, 11, 10) fused, n = 9 alone at L = 1320
    ((16, 20, 19), 2, 2),       # n = 19 at L = 320 (64-aligned) takes the TMA tensor-core pass
    ((19, 19, 19, 19), 1, 4),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("shape,nrhs,fib", CASES)
def test_mixed_solve_through_fibre_passes(shape, nrhs, fib):
    p = si.random_problem(shape, nrhs=nrhs, seed=sum(shape) + nrhs)
    plan = Plan(A=p.A, nrhs=nrhs, prec="mixed")
    d = plan.describe()
    assert d["transform_fib_passes"] == fib, d
    Xd, info = plan.solve(to_device(p.B), info=True)
    torch.cuda.synchronize()
    assert info["status"] == 0, info
    assert info["refine_iters"] >= 1
    X = from_device(Xd, p.B.shape)
    assert oracle.rel_err(X, oracle.solve(p.A, p.B)) < TOL


def test_forward_transform_matches_mode_products():
    """One forward transform on its own: Y = B x_1 U_1^* ... x_N U_N^* with the
    plan's own Schur vectors, against the oracle's mode products (FP32 pass:
    relative error at the FP32 rounding level of n-term sums)."""
    shape = (23, 9, 17)
    p = si.random_problem(shape, nrhs=1, seed=5)
    plan = Plan(A=p.A, nrhs=1, prec="mixed")
    assert plan.describe()["transform_fib_passes"] == 3
    B = p.B                                   # shape + (1,): one right-hand side
    T = to_device(B, dtype=torch.complex64)
    plan.forward(T)
    torch.cuda.synchronize()
    Y = from_device(T, B.shape)
    ref = B.copy()
    for j in range(len(shape)):
        Q, _ = plan.factors(j)
        ref = oracle.mode_product(Q.conj().T, ref, j)
    err = np.max(np.abs(Y - ref)) / np.max(np.abs(ref))
    assert err < 5e-6, err
