"""sylv_sweep_static: the sweep for callers that cannot allocate device memory.

Some callers run with all device memory already reserved by another
allocator, or inside a loop where a cudaMalloc would stall on an implicit
device synchronisation; for them the library keeps the sweep's scratch in a
fixed array of its own.  This test calls that entry point through the C ABI
and compares it with the workspace-based sylv_sweep, twice in a row (the
array keeps the previous call's contents, which must not leak into the next
result).  It is collected last so that a failure here leaves every other test
already run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import sylv_inputs as si
from paper_2412_15840_gb300 import Plan, SylvError, from_device, to_device
from paper_2412_15840_gb300.build import build

pytestmark = pytest.mark.gpu

# per-phase tolerances used by the other sweep tests (relative max-norm)
TOL = {"fp64": 1e-13, "mixed": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    build()
    assert torch.cuda.is_available()


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape,nrhs", [((8, 8, 8), 1), ((17, 11, 9), 2), ((13, 1, 9, 4), 3)])
def test_static_sweep_matches_workspace_sweep_twice(shape, nrhs, prec):
    p = si.random_problem(shape, nrhs, seed=17 + len(shape))
    plan = Plan(A=p.A, nrhs=nrhs, prec=prec)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    C = to_device(p.B, dtype=dt)
    ref = from_device(plan.sweep(C.clone()), p.B.shape)
    for _ in range(2):
        Y = plan.sweep_static(C.clone())
        torch.cuda.synchronize()
        assert rel(from_device(Y, p.B.shape), ref) < TOL[prec]


def test_static_sweep_alternating_plans_and_limit():
    # two plans of different tile counts share the array one after the other
    pa = si.random_problem((9, 10, 11), 1, seed=3)
    pb = si.random_problem((2,) * 12, 2, seed=4, shift=2.0)
    plans = [(Plan(A=pa.A, nrhs=1), pa), (Plan(A=pb.A, nrhs=2), pb)]
    for plan, p in plans + plans:
        C = to_device(p.B)
        ref = from_device(plan.sweep(C.clone()), p.B.shape)
        out = from_device(plan.sweep_static(C.clone()), p.B.shape)
        assert rel(out, ref) < TOL["fp64"]
    # a sweep whose tile counters exceed the fixed array is refused
    big = Plan(A=[np.array([[2.0 + 0j]])] + [np.eye(2) * 3 + 0j] * 20, nrhs=1, block=[1] * 21)
    with pytest.raises(SylvError) as e:
        big.sweep_static(torch.zeros(2 ** 20, dtype=torch.complex128, device="cuda"))
    assert e.value.status == 2
