"""Parity of the sm_103a library (through its C ABI) with the FP64 CPU oracle.

Tolerances (relative max-norm error against the oracle's X):
  SYLV_FP64         1e-12
  SYLV_MIXED_FP32   1e-10   (after FP64 residual refinement)
Per-phase checks hand the oracle the plan's own Schur factors (a Schur form
is not unique, the solution is)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import sylv_inputs as si
from paper_2412_15840_gb300 import Plan, SylvError, from_device, to_device
from paper_2412_15840_gb300.build import build

from gpu_helpers import sampled_residual

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-10}
# sampled backward error bound: FP64 rounding level, or the refinement target / 10
ETA = {"fp64": 1e-14, "mixed": 1e-11}
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def built():
    build()
    assert torch.cuda.is_available()


def gpu_solve(A, B, prec, **kw):
    nrhs = B.shape[-1]
    plan = Plan(A=A, nrhs=nrhs, prec=prec, **kw)
    Bd = to_device(B)
    Xd, info = plan.solve(Bd, info=True)
    torch.cuda.synchronize()
    return from_device(Xd, B.shape), info, plan


# --------------------------------------------------------------- N=3, n=8 --

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cube_n8_N3(prec):
    p = si.cube_n8_N3()
    X, info, _ = gpu_solve(p.A, p.B, prec)
    assert info["status"] == 0, info
    Xo = oracle.solve(p.A, p.B)
    rows = np.loadtxt(os.path.join(GOLDEN, "cube_n8_N3_X.txt"))
    Xg = (rows[:, 0] + 1j * rows[:, 1]).reshape(p.B.shape, order="F")
    assert oracle.rel_err(X, Xo) < TOL[prec]
    assert oracle.rel_err(X, Xg) < TOL[prec]
    if prec == "mixed":
        assert info["refine_iters"] >= 1


# ------------------------------------------------------ shapes, edge cases --

SHAPES = [
    ((5,), 1), ((7,), 3), ((1,), 2), ((1, 1, 1), 1), ((3, 4), 1), ((13, 9), 2),
    ((2, 1, 3), 1), ((1, 6, 1, 5), 2), ((8, 8, 8), 1), ((17, 11, 9), 2),
    ((33, 5, 7), 1), ((2, 2, 2, 2, 2, 2, 2, 2, 2, 2), 1), ((3, 1, 4, 1, 5, 2), 3),
    ((70, 3), 1), ((9, 10, 11, 3), 1), ((100, 2, 2), 1),
    # modes longer than the largest automatic tile extent (64)
    ((600, 9), 1), ((130, 3, 2), 2),
    # first mode on the tensor cores (n % 8 == 0, 32 <= n <= 80, >= 64 columns)
    ((64, 70), 1), ((48, 5, 16), 2), ((80, 9, 8), 1), ((32, 32, 32), 1), ((40, 2, 33), 2),
    # later modes on the tensor cores with fewer than 64 rows before them (tiles of
    # the flattened (l, r) index; odd L takes the 8-byte loads)
    ((48, 40, 3), 2), ((9, 33, 2), 3), ((12, 5, 48), 1),
    # 16 <= n < 32 on the tensor cores (K padded to 8, N to 16)
    ((19, 19, 19), 1), ((16, 17, 23), 2), ((24, 9, 21), 1),
]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape,nrhs", SHAPES)
def test_shapes_vs_oracle(shape, nrhs, prec):
    p = si.random_problem(shape, nrhs, seed=sum(shape) + nrhs)
    X, info, _ = gpu_solve(p.A, p.B, prec)
    assert info["status"] == 0, info
    assert oracle.rel_err(X, oracle.solve(p.A, p.B)) < TOL[prec]


@pytest.mark.parametrize("block", [(1, 1, 1), (2, 3, 4), (5, 1, 2), (17, 1, 1), (3, 11, 9),
                                   (17, 11, 9)])
def test_sweep_tiling_does_not_change_the_result(block):
    p = si.random_problem((17, 11, 9), 2, seed=4)
    Xo = oracle.solve(p.A, p.B)
    for prec in ("fp64", "mixed"):
        X, info, _ = gpu_solve(p.A, p.B, prec, block=block)
        assert info["status"] == 0
        assert oracle.rel_err(X, Xo) < TOL[prec]


def test_in_place_fp64():
    p = si.random_problem((12, 7, 5), 2, seed=8)
    plan = Plan(A=p.A, nrhs=2, prec="fp64")
    Bd = to_device(p.B)
    plan.solve(Bd, X=Bd)
    X = from_device(Bd, p.B.shape)
    assert oracle.rel_err(X, oracle.solve(p.A, p.B)) < TOL["fp64"]


def test_given_schur_factors():
    p = si.random_problem((9, 6, 4), 1, seed=9)
    f = oracle.schur_factors(p.A)
    Q = [u if u is not None else np.eye(1) for u, _ in f]
    T = [t for _, t in f]
    for prec in ("fp64", "mixed"):
        plan = Plan(Q=Q, T=T, nrhs=1, prec=prec)
        X = from_device(plan.solve(to_device(p.B)), p.B.shape)
        assert oracle.rel_err(X, oracle.solve(p.A, p.B)) < TOL[prec]


def test_errors_are_reported():
    A = [np.diag([1.0 + 0j, 2.0]), np.diag([-1.0 + 0j, 5.0])]
    with pytest.raises(SylvError) as e:
        Plan(A=A, nrhs=1)
    assert e.value.status == 3                      # SYLV_ERR_SINGULAR
    with pytest.raises(SylvError) as e:
        Plan(A=[np.eye(3)], nrhs=0)
    assert e.value.status == 2                      # SYLV_ERR_SHAPE
    p = si.random_problem((6, 5), 1, seed=1)
    plan = Plan(A=p.A, nrhs=1, prec="mixed")
    Bd = to_device(p.B)
    with pytest.raises(SylvError) as e:
        plan.solve(Bd, X=Bd)
    assert e.value.status == 1                      # mixed cannot run in place
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(SylvError) as e:
        plan.solve(Bd, workspace=small)
    assert e.value.status == 9                      # SYLV_ERR_WORKSPACE


# ---------------------------------------------------------------- per phase --

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(8, 8, 8), (13, 1, 9, 4), (2, 2, 3, 2, 2), (64, 70),
                                   (48, 5, 16), (40, 2, 33), (80, 9, 8), (48, 40, 3),
                                   (9, 33, 2), (2,) * 7, (2,) * 14, (3, 2, 2, 2, 2, 2),
                                   (19, 19, 19), (16, 17, 23)])
def test_phases_with_the_plans_factors(shape, prec):
    p = si.random_problem(shape, 2, seed=len(shape))
    plan = Plan(A=p.A, nrhs=2, prec=prec)
    U, T = [], []
    for j in range(len(shape)):
        Qj, Tj = plan.factors(j)
        U.append(None if shape[j] == 1 else Qj)
        T.append(Tj)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    tol = 1e-13 if prec == "fp64" else 2e-5
    C_o = oracle.forward_transform(U, p.B)
    C_g = from_device(plan.forward(to_device(p.B, dtype=dt)), p.B.shape)
    assert oracle.rel_err(C_g, C_o) < tol
    Y_o = oracle.triangular_sweep(T, C_o)
    Y_g = from_device(plan.sweep(to_device(C_o, dtype=dt)), p.B.shape)
    assert oracle.rel_err(Y_g, Y_o) < tol
    X_o = oracle.back_transform(U, Y_o)
    X_g = from_device(plan.back(to_device(Y_o, dtype=dt)), p.B.shape)
    assert oracle.rel_err(X_g, X_o) < tol
    # FP64 residual of a perturbed solution
    Xp = X_o + 1e-3 * si.complex_gaussian(np.random.default_rng(3), X_o.shape)
    R_o = oracle.residual(p.A, Xp, p.B)
    R_g = from_device(plan.residual(to_device(p.B), to_device(Xp)), p.B.shape)
    scale = sum(np.abs(a).sum(axis=1).max() for a in p.A) * np.abs(Xp).max() + np.abs(p.B).max()
    assert np.abs(R_g - R_o).max() < 1e-14 * scale


# --------------------------------------------------- the benchmark workloads --

@pytest.fixture(scope="module")
def n64_N4():
    p = si.cube_n64_N4()
    return p, oracle.solve(p.A, p.B)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cube_n64_N4_full_size(n64_N4, prec):
    p, Xo = n64_N4
    X, info, _ = gpu_solve(p.A, p.B, prec)
    assert info["status"] == 0, info
    assert oracle.rel_err(X, Xo) < TOL[prec]


def test_binary_N29_reduced_vs_oracle():
    # same structure as the N=29 workload: 2x2 operators + 2I, singletons [1.5]
    shape = tuple(1 if j in (5, 13) else 2 for j in range(1, 19))
    p = si.random_problem(shape, 1, seed=0, shift=2.0, scale=1 / np.sqrt(2))
    Xo = oracle.solve(p.A, p.B)
    for prec in ("fp64", "mixed"):
        X, info, _ = gpu_solve(p.A, p.B, prec)
        assert info["status"] == 0
        assert oracle.rel_err(X, Xo) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_binary_N29_full_size_sampled_residual(prec):
    p = si.binary_N29()
    plan = Plan(A=p.A, nrhs=1, prec=prec)
    Bd = to_device(p.B)
    Xd, info = plan.solve(Bd, info=True)
    assert info["status"] == 0, info
    eta = sampled_residual(p.A, p.B.reshape(-1, order="F"), Xd, p.shape, 1)
    assert eta < ETA[prec]


def test_advdiff_n48_mixed_vs_fft_closed_form():
    p = si.advdiff_n48()
    X, info, _ = gpu_solve(p.A, p.B, "mixed")
    assert info["status"] == 0, info
    n = 48
    h = 2 * np.pi / n
    w = 2 * np.pi * np.arange(n) / n
    lam = 0.01 * (2 * np.cos(w) - 2) / h ** 2 + 0.5 * (1j * np.sin(w)) / h + 1.0
    Lam = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    Xf = np.fft.ifftn(np.fft.fftn(p.B, axes=(0, 1, 2)) / Lam[..., None], axes=(0, 1, 2))
    assert oracle.rel_err(X, Xf) < TOL["mixed"]


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cube_n19_N7_full_size_sampled_residual(prec):
    p = si.cube_n19_N7()
    plan = Plan(A=p.A, nrhs=1, prec=prec)
    Bd = to_device(p.B)
    Bflat = p.B.reshape(-1, order="F")
    del p.B
    Xd, info = plan.solve(Bd, info=True)
    assert info["status"] == 0, info
    eta = sampled_residual(p.A, Bflat, Xd, p.shape, 1, count=1000)
    assert eta < ETA[prec]
