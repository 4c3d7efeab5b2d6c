"""Benchmark: solved entries/s of the N-dimensional Sylvester solver on GB300.

Workload (one step = one full solve, all hot-path phases): N=4, n_k=64
(16,777,216 complex entries, 268 MB per complex128 tensor), operators
A_k = (randn + i randn)/8 + 3I, complex Gaussian B, seed = rank.  The headline
`value` is the mixed path (FP32 transforms and sweep, FP64 residual and
update, refinement to 1e-10 relative error); the plain FP64 path is reported
beside it.  The Schur setup (plan creation) is outside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank solves its own equation (independent problems, weak
scaling); timings are the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import sylv_inputs as si  # noqa: E402

METRIC = "entries solved/s, FP64 vs mixed+refine at 1e-10 rel err; % of roofline"
UNIT = "entries/s"
SHAPE = (64, 64, 64, 64)
RTOL = 1e-10
MAX_REFINE = 3

# FP64 FMA pipe: 2 FP64 FMA per clock per SM (152 SMs) at the 2070 MHz
# maximum SM clock -> 152 * 2 * 2 * 2.07e9 = 1.2586e12 FLOP/s
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12

# DRAM traffic per launch of the FP64 residual pass kernel, from an ncu capture
# (see profiles/); valid only for the kernel source it was measured on.
TRAFFIC = {"kernels_sha": "5fe5f836f06544a9", "bytes_per_launch": 761.8e6,
           "source": "profiles/kernels_N4_n64.md (mean of the 4 residual-pass launches)"}


def kernels_sha() -> str:
    p = os.path.join(ROOT, "paper_2412_15840_gb300", "csrc", "kernels.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-oracle", action="store_true",
                    help="skip the oracle error check and CPU baseline")
    ap.add_argument("--kernels-once", action="store_true",
                    help="run each hot-path kernel family once on the workload (for ncu)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the plans' default tilings (no sylv_plan_autotune)")
    ap.add_argument("--workloads", default="N3_n8,N29_n2,advdiff48,batch512,N7_n19",
                    help="other configurations measured in the default run (comma list; "
                         "'none' skips them)")
    ap.add_argument("--workload", default="n64_N4",
                    choices=["n64_N4", "batch512", "advdiff48", "n2_N29", "n19_N7",
                             "evolve_n64_N4", "real_n64_N4"],
                    help="n64_N4 is the benchmark line; the others measure the other "
                         "synthetic workloads (one JSON line each)")
    return ap.parse_args()


def oracle_threads() -> int:
    """Host threads the oracle's mode products use (OpenMP over all cores; its
    sweep is one sequential pass)."""
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n and n.isdigit() else (os.cpu_count() or 1)


# --------------------------------------------------------------- clocks ----

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.active = False
        self.label = "headline"

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            if self.active:
                self.lines.append((self.label, line.strip()))

    def mark(self, on: bool, label: str = "headline"):
        self.label = label
        self.active = on

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return self.summary("headline")

    def summary(self, label: str):
        rows = [l.split(", ") for lab, l in self.lines if lab == label and l.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "power_w_max": max(pw) if pw else None, "samples": len(rows)}


# ------------------------------------------------------------- reference ---

def run_reference(args, rank: int, world: int):
    """The oracle as it stands, on the host cores: one full solve per step."""
    if rank != 0:
        return 0
    import oracle
    p = si.random_problem(SHAPE, 1, seed=0, name="N4_n64")
    entries = p.n_tot * p.nrhs
    for _ in range(args.warmup):
        oracle.solve(p.A, p.B)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.solve(p.A, p.B)
    dt = time.perf_counter() - t0
    value = entries * args.steps / dt
    cores = oracle_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "config": config_block(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "one full CPU-oracle solve of the N=4, n=64 workload per "
                                   "step (C mode products over the host cores, "
                                   "single-thread C sweep)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_block():
    return {"workload": "N4_n64: N=4, n_k=64, 16,777,216 complex entries, 1 RHS, "
                        "A_k=(randn+i randn)/8+3I, seed=rank",
            "N": 4, "n": 64, "nrhs": 1, "entries": 64 ** 4, "rtol": RTOL,
            "prec_headline": "mixed_fp32 (FP32 solve + FP64 residual refinement)",
            "l2": "inputs larger than L2 (268 MB complex128 tensors, 129 MB L2)"}


# ------------------------------------------------------------------- ours --

def sampled_eta(A, B_flat, X_dev, shape, nrhs, count=1000, seed=11):
    """Backward error at sampled entries: r_i = b_i - sum_j sum_k a_{j,i_j k} x_{..k..},
    eta = max|r_i| / (sum_j ||A_j||_inf ||X||_inf + ||B||_inf)  (host arithmetic)."""
    import torch
    rng = np.random.default_rng(seed)
    N = len(shape)
    S = np.cumprod((1,) + tuple(shape[:-1]), dtype=np.int64)
    ntot = int(np.prod(shape, dtype=np.int64))
    ii = np.stack([rng.integers(0, shape[j], size=count) for j in range(N)], axis=1)
    lin = (ii * S).sum(axis=1) + rng.integers(0, nrhs, size=count) * ntot
    acc = np.zeros(count, dtype=np.complex128)
    for j in range(N):
        idx = lin[:, None] + (np.arange(shape[j])[None, :] - ii[:, j:j + 1]) * S[j]
        xs = X_dev[torch.as_tensor(idx.reshape(-1), device=X_dev.device)].cpu().numpy()
        acc += np.einsum("ck,ck->c", A[j][ii[:, j], :], xs.reshape(count, shape[j]))
    r = B_flat[lin] - acc
    an = sum(float(np.abs(a).sum(axis=1).max()) for a in A)
    return float(np.abs(r).max()) / (an * float(X_dev.abs().max().item()) + float(np.abs(B_flat).max()))


def other_workload(args, local: int) -> int:
    """One JSON line for a non-default synthetic workload (both precisions)."""
    import torch
    from paper_2412_15840_gb300.build import build
    build()
    from paper_2412_15840_gb300 import (Plan, from_device, solve_batched, to_device,
                                        workspace_size_batched)
    import oracle
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    import torch.distributed as dist
    from paper_2412_15840_gb300.dist import max_over_ranks, shard, sum_over_ranks
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=dev)
    name = args.workload
    if name == "batch512":
        probs = si.uneven_batch(512, 4, seed=0)
        desc = "512 N=3 equations, n_k ~ U{16..96} (seed 0), A=(randn+i randn)/sqrt(n)+3I, 4 RHS"
    elif name == "advdiff48":
        probs = [si.advdiff_n48()]
        desc = "N=3, n=48 periodic advection-diffusion (0.01 D2 + 0.5 D1 + I), 32 RHS"
    elif name == "n2_N29":
        probs = [si.binary_N29()]
        desc = "N=29, n=2 (modes 5, 17 singletons [1.5]), 2x2 (randn+i randn)/sqrt(2)+2I, 2^27"
    else:
        probs = [si.cube_n19_N7()]
        desc = "N=7, n=19 (893,871,739 entries), A=(randn+i randn)/sqrt(19)+3I"
    if name == "batch512" and world > 1:
        # independent equations: each rank solves its share, no data-path collective
        mine = shard([float(p.n_tot * p.nrhs) for p in probs], rank, world)
        probs = [probs[e] for e in mine]
    # other workloads: one equation does not split across GPUs, every rank
    # solves its own replica
    entries_local = sum(p.n_tot * p.nrhs for p in probs)
    entries = int(sum_over_ranks(entries_local, device=dev))
    Bs = [to_device(p.B, device=dev) for p in probs]
    out = {"workload": name, "description": desc, "entries": entries, "equations": len(probs)}
    stream = torch.cuda.current_stream(dev)
    for prec in ("mixed", "fp64", "mixed_emu"):
        t0 = time.perf_counter()
        plans = [Plan(A=p.A, nrhs=p.nrhs, prec=prec, rtol=RTOL, max_refine=MAX_REFINE,
                      device=local) for p in probs]
        setup = time.perf_counter() - t0
        Xs = [torch.empty_like(b) for b in Bs]
        ws = torch.empty(max(256, workspace_size_batched(plans)), dtype=torch.uint8, device=dev)

        def step():
            solve_batched(plans, Bs, Xs, ws, stream=stream)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, device=dev)
        infos = solve_batched(plans, Bs, Xs, ws, stream=stream, info=True)
        rec = {"ms_per_step": ms, "value": entries / (ms * 1e-3), "setup_s": setup,
               "max_refine_iters": max(i["refine_iters"] for i in infos),
               "status": sorted({i["status"] for i in infos})}
        if prec == "mixed_emu":
            rec["tensor_core_residual_equations"] = sum(
                1 for i in infos if i["tensor_core_residual"])
        if name in ("batch512", "advdiff48"):
            pick = [min(range(len(probs)), key=lambda e: probs[e].n_tot)] if name == "batch512" \
                else [0]
            if name == "batch512":
                pick += [1, 2]
            rec["rel_err_vs_oracle_max"] = max(
                oracle.rel_err(from_device(Xs[e], probs[e].B.shape),
                               oracle.solve(probs[e].A, probs[e].B)) for e in pick)
            rec["oracle_checked_equations"] = pick
        else:
            p = probs[0]
            rec["sampled_backward_error"] = sampled_eta(p.A, p.B.reshape(-1, order="F"), Xs[0],
                                                        p.shape, p.nrhs)
        out[prec] = rec
        del plans, Xs, ws
        torch.cuda.empty_cache()
    line = {"metric": METRIC, "unit": UNIT, "value": out["mixed"]["value"], "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak" if name == "batch512" else "replicas only",
            "data": "synthetic", "config": out}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def evolve_workload(args, local: int) -> int:
    """Theorem 1 on the N=4, n=64 operators: X(t) at t = 0.1 of
    X_t = sum_j A_j (x)_j X + B from a Gaussian X(0), both precisions."""
    import torch
    from paper_2412_15840_gb300.build import build
    build()
    from paper_2412_15840_gb300 import Plan, from_device, to_device
    import oracle
    from paper_2412_15840_gb300.dist import max_over_ranks
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=dev)
    p = si.cube_n64_N4()
    X0 = si.initial_state(p.shape, 1, seed=1)
    t = 0.1
    Bd, X0d = to_device(p.B, device=dev), to_device(X0, device=dev)
    entries = p.n_tot * world
    out = {"workload": "evolve_n64_N4",
           "description": "Theorem 1: X(0.1) of X_t = sum_j A_j (x)_j X + B, N=4, n_k=64, "
                          "A=(randn+i randn)/8+3I, B and X(0) unit complex Gaussian",
           "entries": entries, "t": t}
    ref = None if args.no_oracle else oracle.evolve(p.A, p.B, X0, t)
    stream = torch.cuda.current_stream(dev)
    for prec in ("mixed", "fp64", "mixed_emu"):
        plan = Plan(A=p.A, nrhs=1, prec=prec, rtol=RTOL, max_refine=MAX_REFINE, device=local)
        X = torch.empty_like(Bd)
        ws = torch.empty(plan.evolve_workspace_bytes(), dtype=torch.uint8, device=dev)
        plan.set_timing(True)
        for _ in range(args.warmup):
            plan.evolve(t, Bd, X0d, X=X, workspace=ws, stream=stream)
        torch.cuda.synchronize(dev)
        plan.timing(reset=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            plan.evolve(t, Bd, X0d, X=X, workspace=ws, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, device=dev)
        tm = plan.timing(reset=True)
        _, info = plan.evolve(t, Bd, X0d, X=X, workspace=ws, stream=stream, info=True)
        rec = {"ms_per_step": ms, "value": entries / (ms * 1e-3),
               "phase_ms": {k: v / max(1, tm["solves"]) for k, v in tm["ms"].items()},
               "refine_iters": info["refine_iters"], "status": info["status"]}
        if ref is not None:
            rec["rel_err_vs_oracle"] = oracle.rel_err(from_device(X, p.B.shape), ref)
        out[prec] = rec
        del plan, X, ws
        torch.cuda.empty_cache()
    line = {"metric": "entries evolved/s (Theorem 1, t = 0.1)", "unit": "entries/s",
            "value": out["mixed"]["value"], "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "replicas only",
            "data": "synthetic", "config": out}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def real_workload(args, local: int) -> int:
    """Real A_j and B (N=4, n=64): the real-arithmetic variant (real Schur factors,
    float64 / float32 tensors) in FP64 and mixed precision, beside the complex
    plan solving the same problem as complex data."""
    import torch
    from paper_2412_15840_gb300.build import build
    build()
    from paper_2412_15840_gb300 import Plan, from_device, to_device
    import oracle
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    import torch.distributed as dist
    from paper_2412_15840_gb300.dist import max_over_ranks
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=dev)
    p = si.real_cube_n64_N4(seed=rank)
    entries = p.n_tot * world
    out = {"workload": "real_n64_N4",
           "description": "N=4, n_k=64, real A=randn/8+3I, real unit Gaussian B, 1 RHS",
           "entries": entries, "l2": "inputs larger than L2 (134 MB float64 tensors)"}
    ref = None
    if not args.no_oracle:
        ref = oracle.solve([a.astype(np.complex128) for a in p.A],
                           p.B.astype(np.complex128)).real
    stream = torch.cuda.current_stream(dev)
    legs = (("real_mixed", "mixed", True), ("real_fp64", "fp64", True),
            ("complex_mixed", "mixed", False), ("complex_fp64", "fp64", False))
    for name, prec, real in legs:
        plan = Plan(A=p.A, nrhs=1, prec=prec, rtol=RTOL, max_refine=MAX_REFINE, device=local,
                    real=real)
        Bd = to_device(p.B if real else p.B.astype(np.complex128), device=dev)
        X = torch.empty_like(Bd)
        ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device=dev)
        plan.set_timing(True)
        for _ in range(args.warmup):
            plan.solve(Bd, X=X, workspace=ws, stream=stream)
        torch.cuda.synchronize(dev)
        plan.timing(reset=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            plan.solve(Bd, X=X, workspace=ws, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, device=dev)
        tm = plan.timing(reset=True)
        _, info = plan.solve(Bd, X=X, workspace=ws, stream=stream, info=True)
        rec = {"ms_per_step": ms, "value": entries / (ms * 1e-3),
               "phase_ms": {k: v / max(1, tm["solves"]) for k, v in tm["ms"].items()},
               "refine_iters": info["refine_iters"], "status": info["status"]}
        if ref is not None:
            Xh = from_device(X, p.B.shape)
            rec["rel_err_vs_oracle"] = oracle.rel_err(Xh.real if not real else Xh, ref)
        out[name] = rec
        del plan, X, ws, Bd
        torch.cuda.empty_cache()
    line = {"metric": METRIC, "unit": UNIT, "value": out["real_mixed"]["value"], "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "data": "synthetic", "dtype": "f32+f64 (real)", "config": out}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def kernels_once(local: int, small_n: bool = False, n19: bool = False) -> int:
    """One launch group of every hot-path kernel family, in this order:
    FP64 residual passes, FP32 forward passes (first mode and modes 2-4 on
    the tensor cores), FP32 sweep, FP32 back passes, FP64 forward passes,
    FP64 sweep, then one solve with the tensor-core residual, then one mixed
    solve of the real-arithmetic variant on real operators of the same shape
    (a short, fixed launch sequence for ncu captures).  With --workload n2_N29:
    the same sequence (without the last two solves) on the n = 2 operators at
    N = 25.  With --workload n19_N7: the sequence up to the tensor-core-residual
    solve on the n = 19 operators at N = 6 (19^6 = 47M entries: the FP32 passes
    with one thread per fibre, the throughput-bound sweep, the emulated
    residual at n = 19; a few GB on the device)."""
    import torch
    from paper_2412_15840_gb300.build import build
    build()
    from paper_2412_15840_gb300 import Plan, to_device
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    if small_n:
        # the small-n workload's operators at N = 25 (2^23 entries, modes 5 and 17
        # singletons): the same kernels per entry as N = 29, few GB for ncu
        shape = tuple(1 if j in (4, 16) else 2 for j in range(25))
        p = si.random_problem(shape, 1, seed=0, shift=2.0, scale=1.0 / np.sqrt(2.0))
    elif n19:
        p = si.random_problem((19,) * 6, 1, seed=0, name="N6_n19")
    else:
        p = si.random_problem(SHAPE, 1, seed=0, name="N4_n64")
    m = Plan(A=p.A, nrhs=1, prec="mixed", device=local)
    f = Plan(A=p.A, nrhs=1, prec="fp64", device=local)
    B = to_device(p.B, device=dev)
    X = B.clone()
    R = torch.empty_like(B)
    W = B.to(torch.complex64)
    m.residual(B, X, R)
    m.forward(W)
    m.sweep(W)
    m.back(W)
    f.forward(X)
    f.sweep(X)
    if not small_n:
        # one solve with the tensor-core residual (k_resid_oz passes)
        e = Plan(A=p.A, nrhs=1, prec="mixed_emu", device=local)
        e.solve(B, torch.empty_like(B))
    if not small_n and not n19:
        # one mixed solve of the real-arithmetic variant (k_modeprod_r, the
        # tensor-core passes on the complex view, k_sweep<float, true>)
        q = si.real_cube_n64_N4()
        r = Plan(A=q.A, nrhs=1, prec="mixed", real=True, device=local)
        Br = to_device(q.B, device=dev)
        r.solve(Br, torch.empty_like(Br))
    torch.cuda.synchronize(dev)
    print("kernels-once ok")
    return 0


# ------------------------------------------------------------ workloads ----
# Every synthetic configuration of the solver's benchmark suite, measured in
# the default run beside the headline: FP64, mixed (FP64 residual) and mixed
# with the tensor-core residual; error against the oracle (or the sampled
# backward error where the oracle would take minutes); the phase split of one
# solve with phase timing on; each phase's achieved rate against its roofline.

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "of fallback (6.8 TB/s)"


def phase_work(prec, desc, shape, E, iters):
    """Work of each phase of one solve of one equation with E entries.

    FP64 phases: flops, the method's count (Section 2.1, complex multiply-add =
    8 flops: 8 n_j per entry and mode for a transform or residual pass,
    4 sum_j (n_j - 1) + 11 for the sweep) and the count the kernels execute
    (Gauss's three-multiplication product, 6 n_j, in the residual and in the
    transform passes of even n_j >= 8).  FP32 and tensor-core phases: bytes of
    the pass model, each of the plan's P passes reading and writing the tensor
    once (complex64: 16 B per entry; +8 where a pass reads or writes
    complex128; the correction's last back pass also reads X: +16); the sweep
    16 B (complex64 in and out), or 32 B in FP64 for the entrywise division of
    Remark 1; a tensor-core residual pass 48 B (X, R in and out)."""
    P = desc["transform_passes"]
    ns = [n for n in shape if n > 1]
    meth = 8 * sum(ns) * E
    exe_t = sum((6 * n if (n >= 8 and n % 2 == 0) else 8 * n) for n in ns) * E
    sweep_f = (4 * sum(n - 1 for n in shape) + 11) * E
    solves = 1 + iters
    w = {}
    if prec == "fp64":
        w["forward"] = ("fp64", meth, exe_t)
        w["back"] = ("fp64", meth, exe_t)
        w["sweep"] = ("hbm", 32 * E, None) if desc["diag_sweep"] else ("fp64", sweep_f, sweep_f)
        return w
    emu = desc["residual_tc"] == 1
    fwd_corr = 16 * P if emu else 16 * P + 8
    w["forward"] = ("hbm", ((16 * P + 8) + fwd_corr * iters) * E, None)
    w["back"] = ("hbm", ((16 * P + 8) + (16 * P + 24) * iters) * E, None)
    w["sweep"] = ("hbm", 16 * E * solves, None)
    if emu:
        w["residual"] = ("hbm", 48 * desc["residual_passes"] * E * iters, None)
    else:
        w["residual"] = ("fp64", meth * iters, 6 * sum(ns) * E * iters)
    return w


def phase_roofline(prec, phases, descs, shapes, entries_per_eq, iters, hbm_gbs):
    """Per-phase achieved rate and fraction of its roofline (summed over the
    equations; `phases` in ms for one solve of each).  FP64 phases against the
    FP64 pipe: `frac` from the executed flops, `frac_method_count` from the
    method's own count (it exceeds 1 where three-multiplication products run);
    the others against HBM with the pass model's bytes."""
    tot = {}
    for d, shp, E in zip(descs, shapes, entries_per_eq):
        for ph, (kind, amt, exe) in phase_work(prec, d, shp, E, iters).items():
            k, a, x = tot.get(ph, (kind, 0.0, 0.0))
            tot[ph] = (kind, a + amt, x + (exe or 0.0))
    out = {}
    for ph, (kind, amt, exe) in tot.items():
        ms = phases.get(ph, 0.0)
        if ms <= 0 or amt <= 0:
            continue
        sec = ms * 1e-3
        if kind == "fp64":
            out[ph] = {"bound": "fp64 pipe", "achieved_tflops": exe / sec / 1e12,
                       "frac": exe / sec / 1e12 / FP64_PEAK_TFLOPS,
                       "frac_method_count": amt / sec / 1e12 / FP64_PEAK_TFLOPS}
        else:
            out[ph] = {"bound": "hbm", "achieved_gbs": amt / sec / 1e9,
                       "frac": amt / sec / 1e9 / hbm_gbs}
    return out


def run_workloads(args, dev, sampler):
    """The other configurations at N = 1 (see the module's workload list)."""
    import torch
    import oracle
    from paper_2412_15840_gb300 import (Plan, from_device, solve_batched, to_device,
                                        workspace_size_batched)
    from paper_2412_15840_gb300.binding import schur as lib_schur
    hbm_gbs, hbm_note = measured_peaks()
    stream = torch.cuda.current_stream(dev)
    res = {"peaks": {"fp64_tflops": FP64_PEAK_TFLOPS, "fp64_note": "derived: 152 SMs x 2 FMA/clk "
                     "x 2 flops x 2070 MHz", "hbm_gbs": hbm_gbs, "hbm_note": hbm_note}}

    def device_gaussian(shape_with_rhs, seed):
        # unit-variance complex Gaussian drawn on the device (torch Philox,
        # seeded): the 19^7 and batched right-hand sides are too large to draw
        # on the host within the benchmark's time
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        total = int(np.prod(shape_with_rhs, dtype=np.int64))
        v = torch.randn(2 * total, generator=g, device=dev, dtype=torch.float64)
        v.mul_(1.0 / np.sqrt(2.0))
        return torch.view_as_complex(v.view(total, 2))

    def measure(name, probs, Bs, precs, steps, warmup, check, tune=False):
        rec = {}
        shapes = [p.shape for p in probs]
        ents = [p.n_tot * p.nrhs for p in probs]
        entries = sum(ents)
        facs = [[lib_schur(a) if a.shape[0] > 1 else (np.eye(1, dtype=complex), a) for a in p.A]
                for p in probs]
        for prec in precs:
            t0 = time.perf_counter()
            plans = [Plan(Q=[f[0] for f in fa], T=[f[1] for f in fa], nrhs=p.nrhs, prec=prec,
                          rtol=RTOL, max_refine=MAX_REFINE, device=dev.index)
                     for p, fa in zip(probs, facs)]
            setup = time.perf_counter() - t0
            tuned = None
            if tune and len(plans) == 1 and not args.no_autotune:
                t1 = time.perf_counter()
                blk, sweep_ms = plans[0].autotune()
                tuned = {"sweep_block": list(blk), "sweep_ms": sweep_ms,
                         "seconds": time.perf_counter() - t1}
            Xs = [torch.empty_like(b) for b in Bs]
            if len(plans) == 1:
                ws = plans[0].workspace()
                step = lambda: plans[0].solve(Bs[0], Xs[0], workspace=ws, stream=stream)
            else:
                ws = torch.empty(max(256, workspace_size_batched(plans)), dtype=torch.uint8,
                                 device=dev)
                step = lambda: solve_batched(plans, Bs, Xs, ws, stream=stream)
            for _ in range(warmup):
                step()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            sampler.mark(True, name)
            e0.record(stream)
            for _ in range(steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            sampler.mark(False, name)
            ms = e0.elapsed_time(e1) / steps
            if len(plans) == 1:
                _, info = plans[0].solve(Bs[0], Xs[0], workspace=ws, stream=stream, info=True)
                infos = [info]
            else:
                infos = solve_batched(plans, Bs, Xs, ws, stream=stream, info=True)
            r = {"ms_per_solve": ms, "entries_per_s": entries / (ms * 1e-3), "setup_s": setup,
                 "autotuned": tuned,
                 "status": sorted({i["status"] for i in infos}),
                 "refine_iters_max": max(i["refine_iters"] for i in infos)}
            if prec == "mixed_emu":
                r["tensor_core_residual_equations"] = sum(bool(i["tensor_core_residual"])
                                                          for i in infos)
            r.update(check(prec, Xs))
            # phase split: one more solve with phase timing on (a batch then runs
            # its equations one after another instead of under the graph)
            for pl in plans:
                pl.set_timing(True)
            if len(plans) == 1:
                plans[0].solve(Bs[0], Xs[0], workspace=ws, stream=stream)
            else:
                solve_batched(plans, Bs, Xs, ws, stream=stream)
            torch.cuda.synchronize(dev)
            ph = {k: 0.0 for k in ("forward", "sweep", "back", "residual", "update", "total")}
            for pl in plans:
                t = pl.timing(reset=True)
                pl.set_timing(False)
                for k in ph:
                    ph[k] += t["ms"][k]
            r["phase_ms"] = ph
            if len(plans) > 1:
                r["phase_note"] = ("phase_ms sums the equations' phases from one solve with "
                                   "phase timing on, which runs the equations one after another "
                                   "outside the batched graph (single-equation sweeps); the "
                                   "batched time is ms_per_solve")
            iters = r["refine_iters_max"] if prec != "fp64" else 0
            descs = [pl.describe() for pl in plans]
            r["phase_roofline"] = phase_roofline(prec, ph, descs, shapes, ents, iters, hbm_gbs)
            d0 = descs[0]
            r["plan"] = {k: d0[k] for k in ("transform_passes", "transform_tc_passes",
                                            "transform_tma", "transform_group_max",
                                            "residual_passes", "residual_tc", "diag_sweep",
                                            "sweep_block", "sweep_threads", "sweep_ctas_per_sm",
                                            "sweep_lanes", "sweep_tile_levels",
                                            "sweep_far_split", "sweep_3m",
                                            "transform_fib_passes")} \
                if len(plans) == 1 else {
                    "transform_tc_passes": sum(d["transform_tc_passes"] for d in descs),
                    "transform_passes": sum(d["transform_passes"] for d in descs),
                    "diag_sweeps": sum(d["diag_sweep"] for d in descs)}
            rec[prec] = r
            del plans, Xs, ws
            torch.cuda.empty_cache()
        rec["clocks"] = sampler.summary(name)
        rec["entries"] = entries
        return rec

    def oracle_check(probs, picks):
        def check(prec, Xs):
            errs = [oracle.rel_err(from_device(Xs[e], probs[e].B.shape),
                                   oracle.solve(probs[e].A, probs[e].B)) for e in picks]
            return {"rel_err_vs_oracle_max": max(errs), "oracle_checked_equations": len(picks)}
        return check

    def eta_check(p, Bdev):
        def check(prec, Xs):
            return {"sampled_backward_error": sampled_eta_dev(p.A, Bdev, Xs[0], p.shape, p.nrhs)}
        return check

    K = lambda k: max(1, min(args.steps, k))
    W = max(1, min(args.warmup, 2))
    precs = ("fp64", "mixed", "mixed_emu")
    todo = [w.strip() for w in args.workloads.split(",") if w.strip()]

    if "N3_n8" in todo:
        p = si.cube_n8_N3()
        Bs = [to_device(p.B, device=dev)]
        Xo = oracle.solve(p.A, p.B)
        chk = lambda prec, Xs: {"rel_err_vs_oracle": oracle.rel_err(
            from_device(Xs[0], p.B.shape), Xo)}
        res["N3_n8"] = {"config": "N=3, n_k=8 (512 entries), A=(randn+i randn)/sqrt(8)+3I, seed 0"}
        res["N3_n8"].update(measure("N3_n8", [p], Bs, precs, K(20), W, chk, tune=True))
    if "N29_n2" in todo:
        p = si.binary_N29()
        Bd = to_device(p.B, device=dev)
        res["N29_n2"] = {"config": "N=29, n_j=2 except singleton modes 5, 17 ([1.5]); 2x2 "
                         "(randn+i randn)/sqrt(2)+2I; 2^27 entries; seed 0",
                         "error_check": "backward error at 1000 sampled entries"}
        res["N29_n2"].update(measure("N29_n2", [p], [Bd], precs, K(10), W, eta_check(p, Bd),
                                     tune=True))
        del Bd
    if "advdiff48" in todo:
        p = si.advdiff_n48()
        Bs = [to_device(p.B, device=dev)]
        n = 48
        h = 2 * np.pi / n
        w = 2 * np.pi * np.arange(n) / n
        lam = 0.01 * (2 * np.cos(w) - 2) / h ** 2 + 0.5 * (1j * np.sin(w)) / h + 1.0
        Lam = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
        Xf = np.fft.ifftn(np.fft.fftn(p.B, axes=(0, 1, 2)) / Lam[..., None], axes=(0, 1, 2))
        chk = lambda prec, Xs: {"rel_err_vs_fft_closed_form": oracle.rel_err(
            from_device(Xs[0], p.B.shape), Xf)}
        res["advdiff48"] = {"config": "N=3, n=48 periodic advection-diffusion 0.01 D2 + 0.5 D1 "
                            "+ I (h = 2 pi/48), 32 RHS, seed 0; normal operators (Remark 1)",
                            "error_check": "FFT closed form (circulant operators)"}
        res["advdiff48"].update(measure("advdiff48", [p], Bs, precs, K(20), W, chk, tune=True))
    if "batch512" in todo:
        rng, shapes = si.batch_shapes(512, 0)
        probs = [si.Problem(A=[si.gaussian_operator(rng, n, 3.0) for n in shp], B=None,
                            name=f"batch{e}", meta={"shape": shp}) for e, shp in
                 enumerate(shapes)]
        Bs = [device_gaussian(p.meta["shape"] + (4,), 1000 + e) for e, p in enumerate(probs)]
        for p in probs:      # B lives on the device; the host Problem carries the shape
            p.B = np.lib.stride_tricks.as_strided(np.zeros(1, np.uint8), p.meta["shape"] + (4,),
                                                  (0,) * 4)
        big = [e for e, p in enumerate(probs) if max(p.shape) > 80][:6]
        picks = sorted({int(np.argmax([p.n_tot for p in probs])),
                        int(np.argmin([p.n_tot for p in probs]))} | set(big))
        for e in picks:
            probs[e].B = from_device(Bs[e], probs[e].B.shape)
        res["batch512"] = {"config": "512 N=3 equations, n_k ~ U{16..96} (rng.integers, seed "
                           "0), A=(randn+i randn)/sqrt(n)+3I, 4 RHS each, one batched call",
                           "rhs": "drawn on the device (torch Philox, seeds 1000 + e)",
                           "error_check": "oracle on the largest, the smallest and six "
                                          "equations with a mode n > 80"}
        res["batch512"].update(measure("batch512", probs, Bs, precs, K(3), 1,
                                       oracle_check(probs, picks)))
        del Bs
    if "N7_n19" in todo:
        rng = np.random.default_rng(0)
        A = [si.gaussian_operator(rng, 19, 3.0) for _ in range(7)]
        Bd = device_gaussian((19,) * 7 + (1,), 7)
        # B lives on the device only; the host Problem carries the shape
        q = si.Problem(A=A, B=np.lib.stride_tricks.as_strided(np.zeros(1, np.uint8),
                                                               (19,) * 7 + (1,), (0,) * 8))

        def chk(prec, Xs):
            return {"sampled_backward_error": sampled_eta_dev(A, Bd, Xs[0], (19,) * 7, 1)}
        res["N7_n19"] = {"config": "N=7, n=19 (893,871,739 entries), A=(randn+i randn)/sqrt(19)"
                         "+3I (seed 0); B drawn on the device (torch Philox, seed 7)",
                         "error_check": "backward error at 1000 sampled entries"}
        res["N7_n19"].update(measure("N7_n19", [q], [Bd], precs, K(3), 1, chk))
        del Bd
    torch.cuda.empty_cache()
    return res


def sampled_eta_dev(A, B_dev, X_dev, shape, nrhs, count=1000, seed=11):
    """sampled_eta with B on the device (gathered at the sampled entries)."""
    import torch
    rng = np.random.default_rng(seed)
    N = len(shape)
    S = np.cumprod((1,) + tuple(shape[:-1]), dtype=np.int64)
    ntot = int(np.prod(shape, dtype=np.int64))
    ii = np.stack([rng.integers(0, shape[j], size=count) for j in range(N)], axis=1)
    lin = (ii * S).sum(axis=1) + rng.integers(0, nrhs, size=count) * ntot
    acc = np.zeros(count, dtype=np.complex128)
    for j in range(N):
        idx = lin[:, None] + (np.arange(shape[j])[None, :] - ii[:, j:j + 1]) * S[j]
        xs = X_dev[torch.as_tensor(idx.reshape(-1), device=X_dev.device)].cpu().numpy()
        acc += np.einsum("ck,ck->c", A[j][ii[:, j], :], xs.reshape(count, shape[j]))
    b = B_dev[torch.as_tensor(lin, device=B_dev.device)].cpu().numpy()
    r = b - acc
    an = sum(float(np.abs(a).sum(axis=1).max()) for a in A)
    return float(np.abs(r).max()) / (an * float(X_dev.abs().max().item()) +
                                     float(B_dev.abs().max().item()))


def kernels_once_batch(local: int) -> int:
    """One batched mixed solve of 64 equations drawn by the batched workload's
    recipe (64 shape draws, seed 0, 4 RHS): the per-equation passes and one
    k_sweep_batch launch per refinement step (a short sequence for ncu)."""
    import torch
    from paper_2412_15840_gb300.build import build
    build()
    from paper_2412_15840_gb300 import Plan, solve_batched, to_device, workspace_size_batched
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    probs = si.uneven_batch(64, 4, seed=0)
    plans = [Plan(A=p.A, nrhs=4, prec="mixed", device=local) for p in probs]
    Bs = [to_device(p.B, device=dev) for p in probs]
    Xs = [torch.empty_like(b) for b in Bs]
    ws = torch.empty(max(256, workspace_size_batched(plans)), dtype=torch.uint8, device=dev)
    solve_batched(plans, Bs, Xs, ws)
    torch.cuda.synchronize(dev)
    print("kernels-once batch ok")
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.kernels_once:
        if args.workload == "batch512":
            return kernels_once_batch(local)
        return kernels_once(local, small_n=args.workload == "n2_N29",
                            n19=args.workload == "n19_N7")
    if args.workload == "evolve_n64_N4":
        return evolve_workload(args, local)
    if args.workload == "real_n64_N4":
        return real_workload(args, local)
    if args.workload != "n64_N4":
        return other_workload(args, local)

    import torch
    import torch.distributed as dist

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)

    from paper_2412_15840_gb300.build import build
    build()
    from paper_2412_15840_gb300 import Plan, from_device

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_2412_15840_gb300.dist import max_over_ranks as _mor

    def max_over_ranks(x: float) -> float:
        return _mor(x, device=dev)

    p = si.random_problem(SHAPE, 1, seed=rank, name="N4_n64")
    entries = p.n_tot * p.nrhs
    flat = p.B.reshape(-1, order="F")
    B_host = torch.from_numpy(flat).pin_memory()
    B = B_host.to(dev)
    X = torch.empty_like(B)

    t0 = time.perf_counter()
    mixed = Plan(A=p.A, nrhs=1, prec="mixed", rtol=RTOL, max_refine=MAX_REFINE, device=local)
    setup_s_mixed = time.perf_counter() - t0
    t0 = time.perf_counter()
    fp64 = Plan(A=p.A, nrhs=1, prec="fp64", device=local)
    setup_s_fp64 = time.perf_counter() - t0
    tuned = {}
    if not args.no_autotune:
        # tile extents, lanes, CTAs per SM and transform passes chosen by the
        # library's autotuner on this GPU (outside the timed region)
        for nm, pl in (("mixed", mixed), ("fp64", fp64)):
            t1 = time.perf_counter()
            blk, sweep_ms = pl.autotune()
            tuned[nm] = {"sweep_block": list(blk), "sweep_ms": sweep_ms,
                         "seconds": time.perf_counter() - t1}
    ws_m = mixed.workspace()
    ws_f = fp64.workspace()
    stream = torch.cuda.current_stream(dev)

    def timed(fn, k, sampler=None):
        barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if sampler:
            sampler.mark(True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if sampler:
            sampler.mark(False)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / k)

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.5)

    # --- headline: mixed path, device-resident inputs
    def step_mixed():
        mixed.solve(B, X, workspace=ws_m, stream=stream)

    for _ in range(args.warmup):
        step_mixed()
    mixed.set_timing(True)
    ms_mixed = timed(step_mixed, args.steps, sampler)
    mixed.set_timing(False)
    phases_m = mixed.timing(reset=True)
    X_mixed, info_m = mixed.solve(B, X, workspace=ws_m, stream=stream, info=True)
    X_mixed_host = from_device(X_mixed, p.B.shape) if rank == 0 else None
    X_ref_flat = X_mixed.cpu()          # the device solve's result, for the end-to-end check

    # --- plain FP64 path
    X64 = torch.empty_like(B)

    def step_fp64():
        fp64.solve(B, X64, workspace=ws_f, stream=stream)

    for _ in range(args.warmup):
        step_fp64()
    fp64.set_timing(True)
    ms_fp64 = timed(step_fp64, args.steps, sampler)
    fp64.set_timing(False)
    phases_f = fp64.timing(reset=True)
    _, info_f = fp64.solve(B, X64, workspace=ws_f, stream=stream, info=True)
    X_fp64_host = from_device(X64, p.B.shape) if rank == 0 else None

    # --- supplementary: the residual's products on the bf16 tensor cores
    # (SYLV_MIXED_FP32_EMU; not the headline, which keeps the FP64 residual)
    emu = Plan(A=p.A, nrhs=1, prec="mixed_emu", rtol=RTOL, max_refine=MAX_REFINE, device=local)
    if not args.no_autotune:
        t1 = time.perf_counter()
        blk, sweep_ms = emu.autotune()
        tuned["mixed_emu"] = {"sweep_block": list(blk), "sweep_ms": sweep_ms,
                              "seconds": time.perf_counter() - t1}
    ws_e = emu.workspace()
    Xe = torch.empty_like(B)

    def step_emu():
        emu.solve(B, Xe, workspace=ws_e, stream=stream)

    for _ in range(args.warmup):
        step_emu()
    emu.set_timing(True)
    ms_emu = timed(step_emu, args.steps, sampler)
    emu.set_timing(False)
    phases_e = emu.timing(reset=True)
    _, info_e = emu.solve(B, Xe, workspace=ws_e, stream=stream, info=True)
    X_emu_host = from_device(Xe, p.B.shape) if rank == 0 else None
    del ws_e

    # --- end to end through the C ABI: pinned host B -> device, solve, X -> host,
    # every step.  Serial: copy, solve, copy on one stream.  Pipelined (the reported
    # figure): the solves stay in order on `stream`; each step's host-to-device copy
    # runs on one copy stream ahead of its solve and its device-to-host copy on
    # another behind it, with two device buffers, so the copies overlap the
    # neighbouring steps' solves.  Every step's copies are inside the timed region.
    X_host = torch.empty_like(B_host).pin_memory()

    def step_e2e():
        B.copy_(B_host, non_blocking=True)
        mixed.solve(B, X, workspace=ws_m, stream=stream)
        X_host.copy_(X, non_blocking=True)

    for _ in range(args.warmup):
        step_e2e()
    ms_e2e_serial = timed(step_e2e, args.steps, sampler)

    Bd = [B, torch.empty_like(B)]
    Xd = [X, torch.empty_like(B)]
    Bh = [B_host, B_host.clone().pin_memory()]
    Xh = [X_host, torch.empty_like(B_host).pin_memory()]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def pipelined(k):
        e_in = [torch.cuda.Event() for _ in range(2)]
        e_solved = [torch.cuda.Event() for _ in range(2)]
        e_out = [torch.cuda.Event() for _ in range(2)]
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        s_in.wait_event(start)
        s_out.wait_event(start)
        for i in range(k):
            b = i % 2
            if i >= 2:
                s_in.wait_event(e_solved[b])      # the solve that read Bd[b] is done
            with torch.cuda.stream(s_in):
                Bd[b].copy_(Bh[b], non_blocking=True)
            e_in[b].record(s_in)
            stream.wait_event(e_in[b])
            if i >= 2:
                stream.wait_event(e_out[b])       # Xd[b] copied out before it is rewritten
            mixed.solve(Bd[b], Xd[b], workspace=ws_m, stream=stream)
            e_solved[b].record(stream)
            s_out.wait_event(e_solved[b])
            with torch.cuda.stream(s_out):
                Xh[b].copy_(Xd[b], non_blocking=True)
            e_out[b].record(s_out)
        for b in range(2):
            stream.wait_event(e_out[b])
        end.record(stream)
        return start, end

    barrier()
    torch.cuda.synchronize(dev)
    pipelined(args.warmup)
    torch.cuda.synchronize(dev)
    barrier()
    sampler.mark(True)
    t_start, t_end = pipelined(args.steps)
    torch.cuda.synchronize(dev)
    sampler.mark(False)
    barrier()
    ms_e2e = max_over_ranks(t_start.elapsed_time(t_end) / args.steps)
    e2e_matches = bool(torch.equal(Xh[(args.steps - 1) % 2], X_ref_flat))
    clocks = sampler.summary("headline")

    value = world * entries / (ms_mixed * 1e-3)
    value_fp64 = world * entries / (ms_fp64 * 1e-3)
    value_e2e = world * entries / (ms_e2e * 1e-3)
    nbytes = entries * 16

    # roofline of the dominant kernel (FP64 residual passes of the mixed path)
    solves = max(1, phases_m["solves"])
    iters = max(1, info_m["refine_iters"])
    sum_n = sum(n for n in SHAPE if n > 1)
    # one residual over all modes: three FP64 FMAs (6 flops) per entry, mode and k
    # (Gauss's three-multiplication complex product)
    res_flops_per_pass = 6.0 * entries * sum_n
    res_ms = phases_m["ms"]["residual"] / solves          # per solve (all iterations)
    achieved = res_flops_per_pass * iters / (res_ms * 1e-3) / 1e12 if res_ms > 0 else None
    traffic = TRAFFIC["bytes_per_launch"] if TRAFFIC["kernels_sha"] == kernels_sha() else None
    top_phase = max(("forward", "sweep", "back", "residual", "update"),
                    key=lambda k: phases_m["ms"][k])

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "fp32+fp64 (c64 solve, c128 residual)",
        "data": "synthetic", "config": config_block(),
        "fp64": {"value": value_fp64, "unit": UNIT, "ms_per_step": ms_fp64, "dtype": "c128"},
        "speedup_mixed_over_fp64": value / value_fp64,
        "refine_iters": info_m["refine_iters"], "est_rel_err": info_m["est_rel_err"],
        "e2e": {"value": value_e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes, "ms_per_step": ms_e2e,
                "serial_ms_per_step": ms_e2e_serial,
                "overlap": "copies on two copy streams, double-buffered device B and X, "
                           "overlapping the neighbouring steps' solves; solves in order "
                           "on one stream",
                "result_matches_device_solve": e2e_matches},
        "gpu_launches": int(info_m["launches"]) * args.steps,
        "roofline": {"bound": "alu", "kernel": "k_modeprod<double,...,EPI_RESID> (FP64 residual)",
                     "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
                     "traffic": traffic, "traffic_unit": "bytes per launch",
                     "algorithmic_bytes_per_launch": 3 * nbytes,
                     "flops_note": "6 sum(n_j) FP64 flops per entry (3 FMAs per complex term)",
                     "peak_note": "FP64 FMA pipe derived: 152 SMs x 2 FMA/clk x 2 FLOP x 2070 MHz"},
        "phases_ms_per_solve": {
            "mixed": {k: v / solves for k, v in phases_m["ms"].items()},
            "fp64": {k: v / max(1, phases_f["solves"]) for k, v in phases_f["ms"].items()}},
        "top_phase_mixed": top_phase,
        "setup_s": {"mixed": setup_s_mixed, "fp64": setup_s_fp64},
        "clocks": clocks,
        "mixed_emu": {
            "value": world * entries / (ms_emu * 1e-3), "unit": UNIT, "ms_per_step": ms_emu,
            "residual": "mode products on the bf16 tensor cores (exact base-256 digit "
                        "products, FP32-pair sums), not FP64",
            "tensor_core_residual": bool(info_e["tensor_core_residual"]),
            "refine_iters": info_e["refine_iters"],
            "phases_ms_per_solve": {k: v / max(1, phases_e["solves"])
                                    for k, v in phases_e["ms"].items()}},
    }

    hbm_gbs, _ = measured_peaks()
    line["phase_roofline"] = {
        "mixed": phase_roofline("mixed", line["phases_ms_per_solve"]["mixed"], [mixed.describe()],
                                [SHAPE], [entries], info_m["refine_iters"], hbm_gbs),
        "fp64": phase_roofline("fp64", line["phases_ms_per_solve"]["fp64"], [fp64.describe()],
                               [SHAPE], [entries], 0, hbm_gbs),
        "mixed_emu": phase_roofline("mixed_emu", line["mixed_emu"]["phases_ms_per_solve"],
                                    [emu.describe()], [SHAPE], [entries], info_e["refine_iters"],
                                    hbm_gbs)}
    line["plans"] = {"mixed": mixed.describe(), "fp64": fp64.describe(),
                     "mixed_emu": emu.describe(), "autotuned": tuned or None}
    for k in ("mixed", "fp64", "mixed_emu"):
        line["plans"][k]["sweep_block"] = list(line["plans"][k]["sweep_block"])
    del X_mixed, X64, Xe, Bd, Xd, B, X
    torch.cuda.empty_cache()
    if world == 1 and args.workloads not in ("", "none"):
        line["workloads"] = run_workloads(args, dev, sampler)
        line["workloads"]["N4_n64"] = "this line's headline (value, fp64, mixed_emu, " \
                                      "phases_ms_per_solve, phase_roofline)"
    sampler.stop()

    if rank == 0 and not args.no_oracle:
        import oracle
        t0 = time.perf_counter()
        Xo = oracle.solve(p.A, p.B)
        dt = time.perf_counter() - t0
        line["rel_err_vs_oracle"] = {"mixed": oracle.rel_err(X_mixed_host, Xo),
                                     "fp64": oracle.rel_err(X_fp64_host, Xo)}
        line["mixed_emu"]["rel_err_vs_oracle"] = oracle.rel_err(X_emu_host, Xo)
        line["cpu_baseline"] = {
            "value": entries / dt, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
            "sample": "one full CPU-oracle solve of this rank-0 N=4, n=64 equation "
                      "(C mode products over the host cores, single-thread C sweep); "
                      f"{dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
