"""Batched solves (one recorded CUDA graph over forked streams), the sweep
autotuner, and the device-side timeout path (fault injected from the host:
one tile never releases its predecessors, so their bounded waits run out)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import sylv_inputs as si
from paper_2412_15840_gb300 import (Plan, SylvError, from_device, solve_batched, to_device,
                                    workspace_size_batched)
from paper_2412_15840_gb300.build import build

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def built():
    build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def small_batch():
    # the uneven batched workload's recipe at reduced sizes (n_k ~ U{16..40})
    return si.uneven_batch(count=10, nrhs=2, seed=5, lo=16, hi=40)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_graph_matches_oracle_and_replays(small_batch, prec):
    probs = small_batch
    plans = [Plan(A=p.A, nrhs=p.nrhs, prec=prec) for p in probs]
    Bs = [to_device(p.B) for p in probs]
    Xs = [torch.empty_like(b) for b in Bs]
    ws = torch.empty(workspace_size_batched(plans), dtype=torch.uint8, device="cuda")
    infos = solve_batched(plans, Bs, Xs, ws, info=True)
    first = [x.clone() for x in Xs]
    for p, x, inf in zip(probs, Xs, infos):
        assert inf["status"] == 0, inf
        assert oracle.rel_err(from_device(x, p.B.shape), oracle.solve(p.A, p.B)) < TOL[prec]
    # second call with the same arguments replays the recorded graph
    for x in Xs:
        x.zero_()
    solve_batched(plans, Bs, Xs, ws)
    torch.cuda.synchronize()
    for a, b in zip(first, Xs):
        assert torch.equal(a, b)


def test_batched_timing_plans_launch_directly(small_batch):
    probs = small_batch[:3]
    plans = [Plan(A=p.A, nrhs=p.nrhs, prec="fp64") for p in probs]
    plans[1].set_timing(True)
    Bs = [to_device(p.B) for p in probs]
    Xs = [torch.empty_like(b) for b in Bs]
    ws = torch.empty(workspace_size_batched(plans), dtype=torch.uint8, device="cuda")
    infos = solve_batched(plans, Bs, Xs, ws, info=True)
    assert all(i["status"] == 0 for i in infos)
    t = plans[1].timing()
    assert t["solves"] == 1 and t["ms"]["total"] > 0
    for p, x in zip(probs, Xs):
        assert oracle.rel_err(from_device(x, p.B.shape), oracle.solve(p.A, p.B)) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_emu"])
@pytest.mark.parametrize("shape", [(24, 20, 18), (64, 64, 16), (2,) * 12])
def test_autotune_keeps_the_answer(shape, prec):
    # sweep tilings, in-tile lanes, CTAs per SM and the transform passes
    # (tensor cores with or without the TMA pipeline, or CUDA cores) change;
    # the solution may not
    p = si.random_problem(shape, 2, seed=6)
    plan = Plan(A=p.A, nrhs=2, prec=prec)
    block, ms = plan.autotune()
    assert len(block) == len(shape) and ms > 0
    assert all(1 <= b <= n for b, n in zip(block, p.shape))
    d = plan.describe()
    assert tuple(d["sweep_block"]) == tuple(block)
    assert d["sweep_lanes"] in (1, 2, 4) and d["transform_passes"] >= 1
    X = from_device(plan.solve(to_device(p.B)), p.B.shape)
    assert oracle.rel_err(X, oracle.solve(p.A, p.B)) < TOL["mixed" if prec != "fp64" else prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sweep_timeout_is_reported_and_the_context_survives(prec):
    p = si.random_problem((16, 16, 16), 1, seed=7)
    # tile 7 never releases its predecessors: their waits end after 200 ms
    bad = Plan(A=p.A, nrhs=1, prec=prec, block=(4, 4, 4), timeout_ms=200, fault_tile=8)
    with pytest.raises(SylvError) as e:
        bad.solve(to_device(p.B), info=True)
    assert e.value.status == 5                         # SYLV_ERR_TIMEOUT
    torch.cuda.synchronize()
    good = Plan(A=p.A, nrhs=1, prec=prec)
    Xg = from_device(good.solve(to_device(p.B)), p.B.shape)
    assert oracle.rel_err(Xg, oracle.solve(p.A, p.B)) < TOL[prec]
