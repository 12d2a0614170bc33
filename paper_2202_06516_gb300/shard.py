"""Spreading independent instances (sweep members, warm-start cases) over ranks, one process per
GPU, and bringing their per-instance results back to rank 0.

Instances of a batched sweep do not interact, so the data-parallel split needs no collective on
the hot path: each rank advances its own contiguous range of instances with its own batched
solver, and only the small per-instance results (steps, convergence flags, angles, and for the
warm start the equilibrated fields) travel once, at the end, through the process group. This
module holds the host logic only: the partition and the gather.
"""
from __future__ import annotations

from typing import Any, Sequence


def partition(weights: Sequence[float], world: int, rank: int) -> tuple[int, int]:
    """Contiguous range [lo, hi) of instances for `rank` out of `world`, balanced by weight
    (e.g. lattice nodes): instance i goes to the rank whose share of the total weight contains
    the midpoint of i's weight interval. Every instance lands on exactly one rank, ranks hold
    consecutive ranges in rank order, and a rank may receive an empty range when there are fewer
    instances than ranks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need world >= 1 and 0 <= rank < world")
    n = len(weights)
    total = float(sum(weights))
    if n == 0:
        return 0, 0
    if total <= 0:
        weights = [1.0] * n
        total = float(n)
    owner = []
    acc = 0.0
    for w in weights:
        mid = (acc + 0.5 * float(w)) / total
        owner.append(min(world - 1, int(mid * world)))
        acc += float(w)
    lo = next((i for i, o in enumerate(owner) if o >= rank), n)
    hi = next((i for i, o in enumerate(owner) if o > rank), n)
    return lo, hi


def gather(local: list, dist=None) -> list | None:
    """Concatenate every rank's list of per-instance results in rank order on rank 0 (which,
    with `partition`'s contiguous ranges, is instance order); other ranks get None. Without a
    process group (dist None) the local list is returned as is."""
    if dist is None:
        return list(local)
    world = dist.get_world_size()
    parts: list[Any] = [None] * world
    dist.all_gather_object(parts, list(local))
    if dist.get_rank() != 0:
        return None
    out: list = []
    for p in parts:
        out.extend(p)
    return out


def broadcast(obj: Any, dist=None, src: int = 0) -> Any:
    """rank src's object on every rank (identity without a process group)."""
    if dist is None:
        return obj
    box = [obj]
    dist.broadcast_object_list(box, src=src)
    return box[0]


def max_over_ranks(value: float, dist=None) -> float:
    """The largest value over ranks, on every rank (the slowest rank's wall time)."""
    if dist is None:
        return float(value)
    parts: list[Any] = [None] * dist.get_world_size()
    dist.all_gather_object(parts, float(value))
    return float(max(parts))
