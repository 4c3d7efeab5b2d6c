"""Full-size element-wise parity with the FP64 oracle on the two workloads that
are too large for the per-shape tests:

  * N = 29 with n_j = 2 except the singleton modes 5 and 17 (2^27 entries,
    2x2 operators (randn + i randn)/sqrt(2) + 2I, singletons [1.5]): the
    sweep at depth 29, with 17 of its 27 non-singleton modes outside the tile;
  * 512 independent N = 3 equations, n_k ~ U{16..96} (seed 0), 4 right-hand
    sides each, all in one sylv_solve_batched call: tiles of every n in range,
    and the modes above the tensor-core passes' limit.

Every entry of every solution is compared (relative max-norm against the
oracle's X, per equation): 1e-12 for SYLV_FP64, 1e-10 for the mixed path after
refinement.  The oracle solves the 512 equations on the host cores in a thread
pool (its C parts run without the interpreter lock)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import sylv_inputs as si
from paper_2412_15840_gb300 import (Plan, from_device, solve_batched, to_device,
                                    workspace_size_batched)
from paper_2412_15840_gb300.build import build

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def built():
    build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def binary_N29():
    p = si.binary_N29()
    return p, oracle.solve(p.A, p.B)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_binary_N29_full_size_every_entry(binary_N29, prec):
    p, Xo = binary_N29
    assert p.shape[4] == 1 and p.shape[16] == 1 and p.n_tot == 2 ** 27
    plan = Plan(A=p.A, nrhs=1, prec=prec)
    Xd, info = plan.solve(to_device(p.B), info=True)
    assert info["status"] == 0, info
    X = from_device(Xd, p.B.shape)
    del Xd
    assert oracle.rel_err(X, Xo) < TOL[prec]


def _oracle_one(p):
    oracle.set_threads(1)
    return oracle.solve(p.A, p.B)


@pytest.fixture(scope="module")
def batch512():
    probs = si.uneven_batch(512, 4, seed=0)
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        Xo = list(ex.map(_oracle_one, probs))
    return probs, Xo


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch512_one_batched_call_every_equation(batch512, prec):
    probs, Xo = batch512
    assert len(probs) == 512 and all(p.nrhs == 4 for p in probs)
    sizes = [n for p in probs for n in p.shape]
    assert min(sizes) == 16 and max(sizes) == 96 and sum(n > 80 for n in sizes) > 0
    plans = [Plan(A=p.A, nrhs=4, prec=prec) for p in probs]
    Bs = [to_device(p.B) for p in probs]
    Xs = [torch.empty_like(b) for b in Bs]
    ws = torch.empty(max(256, workspace_size_batched(plans)), dtype=torch.uint8, device="cuda")
    infos = solve_batched(plans, Bs, Xs, ws, info=True)
    errs = []
    for p, x, xo, inf in zip(probs, Xs, Xo, infos):
        assert inf["status"] == 0, inf
        errs.append(oracle.rel_err(from_device(x, p.B.shape), xo))
    worst = int(np.argmax(errs))
    assert errs[worst] < TOL[prec], (worst, probs[worst].shape, errs[worst])
