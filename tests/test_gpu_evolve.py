"""sylv_evolve (Theorem 1, Section 3): X(t) of X_t = sum_j A_j (x)_j X + B on
the device, against the oracle's restatement of Eqs. (sylvesterNDC)-(C)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import sylv_inputs as si
from paper_2412_15840_gb300 import Plan, SylvError, from_device, to_device
from paper_2412_15840_gb300.build import build

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def built():
    build()
    assert torch.cuda.is_available()


def _ops(shape, seed, shift=0.0):
    rng = np.random.default_rng(seed)
    A = []
    for n in shape:
        if n == 1:
            A.append(np.array([[1.5 + 0.25j]]))
        else:
            a = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
            A.append(a + shift * np.eye(n))
    return A, rng


def _tensor(rng, shape):
    return np.asfortranarray((rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
                             / np.sqrt(2))


def _evolve(A, B, X0, t, prec, **kw):
    plan = Plan(A=A, nrhs=B.shape[-1] if B.ndim > len(A) else 1, prec=prec, **kw)
    X, info = plan.evolve(t, to_device(B), to_device(X0), info=True)
    assert info["status"] == 0, info
    return from_device(X, B.shape), info, plan


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_seven_modes_at_t_0_1(prec):
    # the system of Section 5.2: N = 7, 2 x 3 x ... x 8, t = 0.1
    shape = (2, 3, 4, 5, 6, 7, 8)
    A, rng = _ops(shape, 7)
    B, X0 = _tensor(rng, shape), _tensor(rng, shape)
    X, info, _ = _evolve(A, B, X0, 0.1, prec)
    assert oracle.rel_err(X, oracle.evolve(A, B, X0, 0.1)) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape,nrhs,t", [((5, 1, 4), 3, 0.7), ((9, 8, 7), 2, 1.3),
                                          ((2, 2, 2, 2, 2, 2, 2, 2, 2), 1, 0.4),
                                          ((70, 3), 1, 0.25)])
def test_shapes_and_right_hand_sides(shape, nrhs, t, prec):
    A, rng = _ops(shape, sum(shape), shift=1.0)
    full = shape + (nrhs,)
    B, X0 = _tensor(rng, full), _tensor(rng, full)
    X, _, _ = _evolve(A, B, X0, t, prec)
    assert oracle.rel_err(X, oracle.evolve(A, B, X0, t)) < TOL[prec]


def test_only_singleton_modes_is_the_scalar_ode():
    A = [np.array([[0.4 - 0.3j]]), np.array([[-1.1 + 0.2j]])]
    rng = np.random.default_rng(3)
    B, X0 = _tensor(rng, (1, 1, 4)), _tensor(rng, (1, 1, 4))
    lam, t = A[0][0, 0] + A[1][0, 0], 0.9
    exact = np.exp(lam * t) * X0 + (np.exp(lam * t) - 1) / lam * B
    X, _, _ = _evolve(A, B, X0, t, "fp64")
    assert oracle.rel_err(X, exact) < 1e-14


def test_time_zero_repeated_times_and_in_place():
    A, rng = _ops((6, 5, 4), 4, shift=2.0)
    B, X0 = _tensor(rng, (6, 5, 4)), _tensor(rng, (6, 5, 4))
    plan = Plan(A=A, nrhs=1, prec="fp64")
    Bd, X0d = to_device(B), to_device(X0)
    assert oracle.rel_err(from_device(plan.evolve(0.0, Bd, X0d), B.shape), X0) < 1e-13
    for t in (0.5, 1.25, 0.5):                         # new t, new t, the first t again
        X = from_device(plan.evolve(t, Bd, X0d), B.shape)
        assert oracle.rel_err(X, oracle.evolve(A, B, X0, t)) < 1e-12
    Xd = X0d.clone()
    plan.evolve(0.5, Bd, Xd, X=Xd)                     # X overwrites X0
    assert oracle.rel_err(from_device(Xd, B.shape), oracle.evolve(A, B, X0, 0.5)) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_normal_operators_use_the_diagonal_sweep(prec):
    A1 = si.periodic_advdiff_operator(12)
    A = [A1, A1, A1]
    rng = np.random.default_rng(5)
    B, X0 = _tensor(rng, (12, 12, 12, 2)), _tensor(rng, (12, 12, 12, 2))
    X, info, _ = _evolve(A, B, X0, 0.3, prec)
    assert info["diagonal_sweep"]
    assert oracle.rel_err(X, oracle.evolve(A, B, X0, 0.3)) < TOL[prec]


def test_timing_and_errors():
    A, rng = _ops((4, 3), 6, shift=1.0)
    B, X0 = _tensor(rng, (4, 3)), _tensor(rng, (4, 3))
    plan = Plan(A=A, nrhs=1, prec="fp64")
    plan.set_timing(True)
    Bd, X0d = to_device(B), to_device(X0)
    plan.evolve(0.2, Bd, X0d)
    tm = plan.timing()
    assert tm["launches"]["evolve"] >= 3 and tm["ms"]["evolve"] > 0
    with pytest.raises(SylvError) as e:
        plan.evolve(float("nan"), Bd, X0d)
    assert e.value.status == 1
    small = torch.empty(plan.evolve_workspace_bytes() - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(SylvError) as e:
        plan.evolve(0.2, Bd, X0d, workspace=small)
    assert e.value.status == 9
