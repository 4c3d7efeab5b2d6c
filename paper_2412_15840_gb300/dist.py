"""Host-side logic of multi-GPU runs: one process per GPU, independent
equations sharded across ranks with no collective on the data path.

Independent equations (and right-hand sides) are the data-parallel axis of
the solver; one equation is not split across GPUs (its mode products would
need an all-to-all per transform).  A rank solves only its own equations; the
only collectives are a barrier around timed regions and a max-reduction of
the per-rank times.
"""
from __future__ import annotations

from typing import List, Sequence


def shard(costs: Sequence[float], rank: int, world: int) -> List[int]:
    """Indices of the equations rank `rank` solves, balancing the summed cost.

    Greedy longest-processing-time assignment: equations in decreasing cost,
    each to the currently least-loaded rank (ties to the lower rank).  Every
    equation goes to exactly one rank; the result is deterministic.
    """
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    load = [0.0] * world
    owner = [0] * len(costs)
    for e in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[e] = r
        load[r] += costs[e]
    return [e for e in range(len(costs)) if owner[e] == rank]


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar over the default process group (identity when
    no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
