"""Host-side logic of the multi-GPU path.

Samples of a batch are independent problems (separate lens-parameter
proposals, Sect. 2.2.1), so ranks share no data: each rank evaluates the
samples of its shard with its own model.  No collective touches the data
path; afterwards the per-sample chi^2 values are gathered in sample order
(the result a sampler needs) and the timings are reduced (a barrier and a
maximum).  Shards balance the work of uneven grids (node x potential
evaluations dominate) with a deterministic greedy longest-first assignment.
"""
from __future__ import annotations

from typing import List, Sequence


def balanced_shards(work: Sequence[float], world: int) -> List[List[int]]:
    """Partition sample indices into `world` shards of near-equal total work.

    Longest-processing-time-first: samples in decreasing work (ties by index)
    go to the currently lightest shard (ties to the lower rank); each shard is
    returned in increasing sample order.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(work)), key=lambda i: (-work[i], i))
    loads = [0.0] * world
    shards: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        shards[r].append(i)
        loads[r] += work[i]
    return [sorted(s) for s in shards]


def shard_for(work: Sequence[float], rank: int, world: int) -> List[int]:
    return balanced_shards(work, world)[rank]


def reduce_max(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group (identity
    when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_in_order(values: Sequence[float], shard: Sequence[int], n_total: int) -> List[float]:
    """Per-sample results of every rank's shard, placed in sample order.

    ``values[k]`` is this rank's result for sample ``shard[k]``.  Every rank
    receives the full list of ``n_total`` values (an all-gather of the
    (index, value) pairs; with one process it is a plain reorder).  Each
    sample must belong to exactly one shard.
    """
    import torch.distributed as dist
    if len(values) != len(shard):
        raise ValueError("one value per sample of the shard")
    pairs = [(int(i), float(v)) for i, v in zip(shard, values)]
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, pairs)
    else:
        parts = [pairs]
    out: List[float] = [float("nan")] * n_total
    seen = [False] * n_total
    for part in parts:
        for i, v in part:
            if not 0 <= i < n_total or seen[i]:
                raise ValueError(f"sample {i} out of range or in two shards")
            seen[i] = True
            out[i] = v
    if not all(seen):
        raise ValueError("some samples belong to no shard")
    return out
