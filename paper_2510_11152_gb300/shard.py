"""Assignment of independent solves to GPUs (one process per GPU).

Independent problems (the batched workload: problems of uneven grid sizes) need no data exchange
between GPUs: each rank solves its share and the reports are gathered once. The assignment balances
the work, which is proportional to the cells of a problem (every problem takes a similar number of
cycles to the same relative tolerance): largest first, each to the rank with the least work so far
(ties to the lowest rank), so every rank's load is within the largest problem of the mean.
"""
from __future__ import annotations


def partition(cells: list[int], world: int) -> list[list[int]]:
    """Indices of `cells` per rank (each list in ascending order), deterministic."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for k in sorted(range(len(cells)), key=lambda i: (-cells[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(k)
        load[r] += cells[k]
    return [sorted(p) for p in parts]


def gather_by_index(local: dict, world: int, count: int, group=None) -> list:
    """Collect {problem index: value} from every rank into one list ordered by problem index (on every
    rank). Uses torch.distributed when world > 1."""
    if world == 1:
        return [local[k] for k in range(count)]
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, local, group=group)
    merged = {}
    for p in parts:
        merged.update(p)
    return [merged[k] for k in range(count)]


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over the ranks (x on every rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
