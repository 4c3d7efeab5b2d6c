"""SYLV_MIXED_FP32_EMU: the refinement residual's mode products on the bf16
tensor cores (exact products of base-256 digits).  The solution must reach the
same 1e-10 relative error against the oracle as the FP64-residual path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import sylv_inputs as si
from paper_2412_15840_gb300 import Plan, from_device, to_device
from paper_2412_15840_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build()
    assert torch.cuda.is_available()


def _solve(A, B, **kw):
    plan = Plan(A=A, nrhs=B.shape[-1], prec="mixed_emu", **kw)
    X, info = plan.solve(to_device(B), info=True)
    return from_device(X, B.shape), info


@pytest.mark.parametrize("shape,nrhs,on_tc", [
    ((64, 64, 64), 1, True),          # first mode and two later modes on the tensor cores
    ((64, 8, 16), 2, True),           # small modes (K padded to 16)
    ((64, 1, 16), 4, True),           # a singleton: sigma folded into the first mode
    ((64, 48), 3, True),
    ((64,), 64, True),                # one mode: the first pass is also the last
    ((64, 24, 1, 8), 1, True),
    ((16, 8, 24, 2), 3, False),       # n = 2: the residual stays FP64
    ((48, 16, 8), 2, True),           # later modes with 48 and 768 rows before them
    ((40, 12, 20), 2, True),          # sizes that are not multiples of 8 (K padded)
    ((64, 24, 9), 1, True),
    ((70, 5), 1, False),              # n = 70 > 64
    ((4, 16, 16), 1, False),          # n = 4 < 8
])
def test_emu_matches_oracle(shape, nrhs, on_tc):
    p = si.random_problem(shape, nrhs, seed=sum(shape) + 3 * nrhs)
    X, info = _solve(p.A, p.B)
    assert info["status"] == 0, info
    assert info["tensor_core_residual"] == on_tc
    assert oracle.rel_err(X, oracle.solve(p.A, p.B)) < 1e-10


def test_emu_residual_accuracy_matches_fp64_residual():
    # one refinement step with each residual: the corrections agree to the
    # residuals' accuracy, far below the FP32 solve's error
    # (the default rtol keeps the conditioning guard satisfied; max_refine = 1 stops
    # both paths after one correction)
    p = si.random_problem((64, 32, 16), 1, seed=21)
    Xe, ie = _solve(p.A, p.B, max_refine=1)
    plan = Plan(A=p.A, nrhs=1, prec="mixed", max_refine=1)
    Xm, im = plan.solve(to_device(p.B), info=True)
    Xm = from_device(Xm, p.B.shape)
    Xo = oracle.solve(p.A, p.B)
    assert ie["tensor_core_residual"] and ie["refine_iters"] == 1
    assert oracle.rel_err(Xe, Xo) < 1e-11 and oracle.rel_err(Xm, Xo) < 1e-11
    assert oracle.rel_err(Xe, Xm) < 1e-11


def test_emu_wide_dynamic_range():
    # entries of B spread over 12 orders of magnitude along the last mode: the
    # digit scale is global, the result is still normwise accurate
    p = si.random_problem((64, 16, 32), 1, seed=22)
    B = p.B * np.logspace(-6, 6, 32)[None, None, :, None]
    X, info = _solve(p.A, B)
    assert info["status"] == 0 and info["tensor_core_residual"]
    assert oracle.rel_err(X, oracle.solve(p.A, B)) < 1e-10


def test_emu_full_size_n64_N4():
    p = si.cube_n64_N4()
    X, info = _solve(p.A, p.B)
    assert info["status"] == 0 and info["tensor_core_residual"] and info["refine_iters"] >= 1
    assert oracle.rel_err(X, oracle.solve(p.A, p.B)) < 1e-10


def test_emu_evolve_and_batched():
    from paper_2412_15840_gb300 import solve_batched, workspace_size_batched
    probs = [si.random_problem((64, 16, 8), 2, seed=30 + e) for e in range(3)]
    plans = [Plan(A=q.A, nrhs=2, prec="mixed_emu") for q in probs]
    Bs = [to_device(q.B) for q in probs]
    Xs = [torch.empty_like(b) for b in Bs]
    ws = torch.empty(workspace_size_batched(plans), dtype=torch.uint8, device="cuda")
    infos = solve_batched(plans, Bs, Xs, ws, info=True)
    for q, x, inf in zip(probs, Xs, infos):
        assert inf["status"] == 0 and inf["tensor_core_residual"]
        assert oracle.rel_err(from_device(x, q.B.shape), oracle.solve(q.A, q.B)) < 1e-10
    q = probs[0]
    X0 = si.initial_state(q.shape, 2, seed=4)
    Xt = from_device(plans[0].evolve(0.2, Bs[0], to_device(X0)), q.B.shape)
    assert oracle.rel_err(Xt, oracle.evolve(q.A, q.B, X0, 0.2)) < 1e-10


def test_emu_ill_conditioned_keeps_the_fp64_residual():
    # eigenvalue sums spread over four decades: kappa 2^-45 would exceed rtol, so the
    # plan keeps the FP64 residual and still reaches 1e-10
    rng = np.random.default_rng(23)
    A = []
    for n in (64, 16, 8):
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        lam = np.geomspace(1e-4, 1.0, n) * np.exp(0.3j * rng.standard_normal(n))
        A.append((Q * lam) @ Q.conj().T)
    B = (rng.standard_normal((64, 16, 8, 1)) + 1j * rng.standard_normal((64, 16, 8, 1)))
    X, info = _solve(A, B, max_refine=8)
    assert info["status"] == 0 and not info["tensor_core_residual"]
    assert oracle.rel_err(X, oracle.solve(A, B)) < 1e-10


@pytest.mark.parametrize("shape,nrhs,t", [((64, 24, 9), 1, 0.3), ((64, 1, 16), 4, 0.7),
                                          ((48, 16, 8), 2, 1.1)])
def test_emu_evolve_on_the_tensor_cores(shape, nrhs, t):
    # Theorem 1 with the right-hand side F formed by digit products (W = B + sum_j
    # A_j (x)_j X0, then the exp(t A_j) products), then the emulated-residual solve
    p = si.random_problem(shape, nrhs, seed=40 + sum(shape))
    X0 = si.initial_state(p.shape, nrhs, seed=41)
    plan = Plan(A=p.A, nrhs=nrhs, prec="mixed_emu")
    X, info = plan.evolve(t, to_device(p.B), to_device(X0), info=True)
    assert info["status"] == 0 and info["tensor_core_residual"]
    ref = oracle.evolve(p.A, p.B, X0, t)
    assert oracle.rel_err(from_device(X, p.B.shape), ref) < 1e-10
