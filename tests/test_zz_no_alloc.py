"""sylv_sweep_static: the sweep for callers that cannot allocate device memory.

Some callers run with all device memory already reserved by another
allocator, or inside a loop where a cudaMalloc would stall on an implicit
device synchronisation; for them the library keeps the sweep's scratch in a
fixed array of its own.  These tests call that entry point through the C ABI
and compare it with the oracle's sweep of Eq. (yi1i2iN) (Algorithm 3 order)
on the plan's own Schur factors, and with the workspace-based sylv_sweep,
twice in a row (the array keeps the previous call's contents, which must not
leak into the next result).  The file is collected last so that a failure
here leaves every other test already run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import sylv_inputs as si
from paper_2412_15840_gb300 import Plan, SylvError, from_device, to_device
from paper_2412_15840_gb300.build import build

pytestmark = pytest.mark.gpu

# per-phase tolerances used by the other sweep tests (relative max-norm): FP64
# rounding, and the complex64 sweep's FP32 rounding over ~sum_j n_j terms
TOL = {"fp64": 1e-13, "mixed": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    build()
    assert torch.cuda.is_available()


def plan_T(plan, shape):
    return [plan.factors(j)[1] for j in range(len(shape))]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape,nrhs", [((8, 8, 8), 1), ((17, 11, 9), 2), ((13, 1, 9, 4), 3)])
def test_static_sweep_matches_oracle_and_workspace_sweep_twice(shape, nrhs, prec):
    p = si.random_problem(shape, nrhs, seed=17 + len(shape))
    plan = Plan(A=p.A, nrhs=nrhs, prec=prec)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    C = to_device(p.B, dtype=dt)
    # the oracle sweeps the same (rounded) right-hand side with the plan's T_j
    Y_o = oracle.triangular_sweep(plan_T(plan, shape), from_device(C, p.B.shape).astype(complex))
    ref = from_device(plan.sweep(C.clone()), p.B.shape)
    assert oracle.rel_err(ref, Y_o) < TOL[prec]
    for _ in range(2):
        Y = plan.sweep_static(C.clone())
        torch.cuda.synchronize()
        Yh = from_device(Y, p.B.shape)
        assert oracle.rel_err(Yh, Y_o) < TOL[prec]
        assert oracle.rel_err(Yh, ref) < TOL[prec]


def test_static_sweep_alternating_plans_and_limit():
    # two plans of different tile counts share the array one after the other
    pa = si.random_problem((9, 10, 11), 1, seed=3)
    pb = si.random_problem((2,) * 12, 2, seed=4, shift=2.0)
    plans = [(Plan(A=pa.A, nrhs=1), pa), (Plan(A=pb.A, nrhs=2), pb)]
    for plan, p in plans + plans:
        C = to_device(p.B)
        Y_o = oracle.triangular_sweep(plan_T(plan, p.shape), p.B)
        ref = from_device(plan.sweep(C.clone()), p.B.shape)
        out = from_device(plan.sweep_static(C.clone()), p.B.shape)
        assert oracle.rel_err(out, Y_o) < TOL["fp64"]
        assert oracle.rel_err(out, ref) < TOL["fp64"]
    # a tiled sweep (non-normal operators) whose 2^20 tile counters exceed the
    # fixed array is refused before anything runs
    shape = (1,) + (2,) * 20
    big = si.random_problem(shape, 1, seed=5, shift=2.0)
    plan = Plan(A=big.A, nrhs=1, block=[1] * len(shape))
    with pytest.raises(SylvError) as e:
        plan.sweep_static(torch.zeros(2 ** 20, dtype=torch.complex128, device="cuda"))
    assert e.value.status == 2
    # the entrywise-division sweep of normal operators needs no tile counters:
    # the same tile count is accepted and matches the oracle
    A = [np.array([[2.0 + 0j]])] + [np.diag([3.0 + 1j, 4.0 - 0.5j])] * 20
    diag = Plan(A=A, nrhs=1, block=[1] * len(shape))
    C = si.complex_gaussian(np.random.default_rng(9), shape + (1,))
    Y = from_device(diag.sweep_static(to_device(C)), C.shape)
    assert oracle.rel_err(Y, oracle.triangular_sweep(plan_T(diag, shape), C)) < TOL["fp64"]
