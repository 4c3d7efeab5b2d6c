"""Parity of the real-arithmetic variant (sylv_plan_create_real) with the
oracle: real Schur factors, real transforms, the quasi-triangular sweep with
its 2 x 2 blocks rotated inside the tiles.  Tolerances as for the complex path
(1e-12 FP64, 1e-10 mixed after refinement); per-phase checks hand the oracle
the plan's own factors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import real_variant as rv
import sylv_inputs as si
from paper_2412_15840_gb300 import Plan, SylvError, from_device, to_device
from paper_2412_15840_gb300.build import build

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def built():
    build()
    assert torch.cuda.is_available()


def _pairs(T):
    return sum(1 for k in range(T.shape[0] - 1) if T[k + 1, k] != 0.0)


def _solve(A, B, prec, **kw):
    plan = Plan(A=A, nrhs=B.shape[-1], prec=prec, real=True, **kw)
    Xd, info = plan.solve(to_device(B), info=True)
    assert Xd.dtype == torch.float64
    return from_device(Xd, B.shape), info, plan


# shift 3 as in the paper's workloads (eigenvalue sums away from zero); most
# modes still hold complex pairs (test_real_cases_hold_complex_pairs)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape,nrhs,shift", [
    ((8, 8, 8), 1, 3.0), ((13, 1, 9, 4), 2, 3.0), ((2, 2, 3, 2, 2), 2, 2.0), ((64, 70), 1, 3.0),
    ((48, 5, 16), 3, 3.0), ((40, 2, 33), 1, 3.0), ((19, 19, 19), 1, 3.0), ((16, 17, 23), 2, 3.0),
    ((7,), 4, 1.0), ((5, 1, 1, 6), 1, 2.0), ((2,) * 6, 1, 2.0), ((3, 2, 2, 2, 2, 2), 1, 2.0),
    ((16,), 3, 2.0), ((12, 1), 70, 2.0), ((128, 6), 1, 3.0), ((36, 24, 4), 2, 3.0)])
def test_real_solve_matches_oracle(shape, nrhs, shift, prec):
    p = si.random_real_problem(shape, nrhs, seed=len(shape) + nrhs, shift=shift)
    X, info, plan = _solve(p.A, p.B, prec)
    assert info["status"] == 0 and info["real"]
    Xo = oracle.solve([a.astype(np.complex128) for a in p.A], p.B.astype(np.complex128))
    assert np.abs(Xo.imag).max() <= 1e-12 * np.abs(Xo).max()
    assert oracle.rel_err(X, Xo.real) < TOL[prec]


def test_real_cases_hold_complex_pairs():
    # the shapes above exercise 2 x 2 blocks (at even offsets) in most modes
    total = 0
    for shape, shift in (((8, 8, 8), 3.0), ((19, 19, 19), 3.0), ((2,) * 6, 2.0)):
        p = si.random_real_problem(shape, 1, seed=len(shape) + 1, shift=shift)
        plan = Plan(A=p.A, nrhs=1, prec="fp64", real=True)
        for j in range(len(shape)):
            Q, T = plan.factors(j)
            assert np.abs(Q.imag).max() == 0.0 and np.abs(T.imag).max() == 0.0
            Q, T = Q.real, T.real
            assert np.abs(Q @ T @ Q.T - p.A[j]).max() < 1e-12 * max(1.0, np.abs(p.A[j]).max())
            assert all(T[k + 1, k] == 0.0 for k in range(1, T.shape[0] - 1, 2))
            total += _pairs(T)
    assert total >= 10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(8, 8, 8), (13, 1, 9, 4), (2, 2, 3, 2, 2), (64, 70),
                                   (40, 2, 33), (19, 19, 19), (2,) * 6])
def test_real_phases_with_the_plans_factors(shape, prec):
    p = si.random_real_problem(shape, 2, seed=len(shape), shift=3.0)
    plan = Plan(A=p.A, nrhs=2, prec=prec, real=True)
    Q, T = [], []
    for j in range(len(shape)):
        Qj, Tj = plan.factors(j)
        Q.append(None if shape[j] == 1 else Qj.real)
        T.append(Tj.real)
    dt = plan.work_dtype
    tol = 1e-13 if prec == "fp64" else 2e-5
    C_o = rv.forward_transform_real(Q, p.B)
    C_g = from_device(plan.forward(to_device(p.B, dtype=dt)), p.B.shape)
    assert oracle.rel_err(C_g, C_o) < tol
    Y_o = rv.quasi_triangular_sweep(T, C_o)
    Y_g = from_device(plan.sweep(to_device(C_o, dtype=dt)), p.B.shape)
    assert oracle.rel_err(Y_g, Y_o) < tol
    X_o = rv.back_transform_real(Q, Y_o)
    X_g = from_device(plan.back(to_device(Y_o, dtype=dt)), p.B.shape)
    assert oracle.rel_err(X_g, X_o) < tol
    # FP64 residual of a perturbed solution
    Xp = X_o + 1e-3 * si.real_gaussian(np.random.default_rng(3), X_o.shape)
    R_o = oracle.residual(p.A, Xp, p.B)
    R_g = from_device(plan.residual(to_device(p.B), to_device(Xp)), p.B.shape)
    scale = sum(np.abs(a).sum(axis=1).max() for a in p.A) * np.abs(Xp).max() + np.abs(p.B).max()
    assert np.abs(R_g - R_o).max() < 1e-14 * scale


@pytest.mark.parametrize("block", [(3, 5, 4), (1, 1, 8), (8, 2, 2), (24, 1, 1)])
def test_real_tilings_keep_pairs_inside_tiles(block):
    # odd or unit extents are widened for modes with 2 x 2 blocks; every tiling
    # gives the same Y as the oracle's quasi-triangular sweep
    p = si.random_real_problem((24, 10, 9), 1, seed=17, shift=3.0)
    plan = Plan(A=p.A, nrhs=1, prec="fp64", real=True, block=block)
    T = [plan.factors(j)[1].real for j in range(3)]
    C = p.B
    Y_g = from_device(plan.sweep(to_device(C, dtype=torch.float64)), C.shape)
    assert oracle.rel_err(Y_g, rv.quasi_triangular_sweep(T, C)) < 1e-13


def test_real_autotune_and_batched():
    from paper_2412_15840_gb300 import solve_batched, workspace_size_batched
    probs = [si.random_real_problem((20 + 4 * e, 12, 6), 2, seed=50 + e, shift=3.0)
             for e in range(3)]
    plans = [Plan(A=q.A, nrhs=2, prec="mixed", real=True) for q in probs]
    plans[0].autotune()
    Bs = [to_device(q.B) for q in probs]
    Xs = [torch.empty_like(b) for b in Bs]
    ws = torch.empty(workspace_size_batched(plans), dtype=torch.uint8, device="cuda")
    infos = solve_batched(plans, Bs, Xs, ws, info=True)
    for q, x, inf in zip(probs, Xs, infos):
        assert inf["status"] == 0 and inf["real"]
        assert oracle.rel_err(from_device(x, q.B.shape), rv.solve_real(q.A, q.B)) < 1e-10


def test_real_full_size_n64_N4():
    p = si.real_cube_n64_N4()
    for prec in ("fp64", "mixed"):
        X, info, _ = _solve(p.A, p.B, prec)
        assert info["status"] == 0
        if prec == "fp64":
            Xo = oracle.solve([a.astype(np.complex128) for a in p.A],
                              p.B.astype(np.complex128)).real
        assert oracle.rel_err(X, Xo) < TOL[prec]


def test_real_plan_rejections():
    p = si.random_real_problem((6, 5), 1, seed=2)
    with pytest.raises(SylvError):
        Plan(A=p.A, nrhs=1, prec="mixed_emu", real=True)
    plan = Plan(A=p.A, nrhs=1, prec="fp64", real=True)
    with pytest.raises((SylvError, ValueError)):
        plan.evolve(0.1, to_device(p.B), to_device(p.B))
    with pytest.raises(ValueError):
        plan.solve(to_device(p.B.astype(np.complex128)))


def test_real_many_coupled_modes():
    # every n = 2 mode holds one complex pair: a tile must hold the whole 2^8 box
    rng = np.random.default_rng(5)
    A = [np.array([[2.0, 1.0], [-1.0, 2.0]]) + 0.1 * rng.standard_normal((2, 2))
         for _ in range(8)]
    B = si.real_gaussian(rng, (2,) * 8 + (1,))
    for prec in ("fp64", "mixed"):
        X, info, plan = _solve(A, B, prec)
        assert info["status"] == 0
        assert all(_pairs(plan.factors(j)[1].real) == 1 for j in range(8))
        assert oracle.rel_err(X, rv.solve_real(A, B)) < TOL[prec]
    # 14 such modes need a 2^14-entry tile: beyond the sweep's tile limit
    with pytest.raises(SylvError):
        Plan(A=A + A[:6], nrhs=1, prec="fp64", real=True)


def test_real_singular_operator_is_refused():
    # eigenvalues +-i in both modes: the sum i + (-i) of the Schur diagonals is zero
    rot = np.array([[0.0, 1.0], [-1.0, 0.0]])
    A = [np.kron(np.eye(2), rot), np.kron(np.eye(3), rot)]
    with pytest.raises(SylvError) as ex:
        Plan(A=A, nrhs=1, prec="fp64", real=True)
    assert "SINGULAR" in str(ex.value)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_real_all_singleton_modes(prec):
    # no mode to transform: X = B / (a_1 + a_2 + a_3)
    A = [np.array([[2.0]]), np.array([[1.5]]), np.array([[-0.25]])]
    B = si.real_gaussian(np.random.default_rng(8), (1, 1, 1, 6))
    X, info, _ = _solve(A, B, prec)
    assert info["status"] == 0
    assert oracle.rel_err(X, B / 3.25) < TOL[prec]
