"""Splitting batched and served work over ranks (one GPU per rank).

Roads of a batch are independent (the paper's "Variations": a parameter
study as embarrassingly parallel jobs), so N ranks take disjoint road ranges
[first, last) of the batch's road table and run them with no communication
on the data path; the results are keyed by road index (each road's draws are
keyed by its own seed and road id), so the union of the ranks' results is
the single-rank result.  A request stream is split the same way, request by
request: rank r serves the requests whose arrival index is r modulo N.
"""
from __future__ import annotations


def road_ranges(work: list[int], world: int) -> list[tuple[int, int]]:
    """Contiguous ranges [first, last) of the roads, one per rank, with about
    equal total work (e.g. cars x steps per road): range r ends at the first
    road where the running total reaches (r + 1) / world of the whole.  Every
    road is in exactly one range; ranges may be empty when roads are fewer
    than ranks."""
    if world < 1:
        raise ValueError("world >= 1")
    n = len(work)
    if any(w < 0 for w in work):
        raise ValueError("work must be non-negative")
    total = sum(work)
    if total == 0:   # nothing to balance: split by count
        return [(r * n // world, (r + 1) * n // world) for r in range(world)]
    ranges = []
    first = 0
    acc = 0
    for r in range(world):
        last = first
        if r == world - 1:
            last = n
        else:
            # take roads while the running total stays within (r + 1) / world
            # of the whole (exact integers)
            while last < n and (acc + work[last]) * world <= (r + 1) * total:
                acc += work[last]
                last += 1
        ranges.append((first, last))
        first = last
    return ranges


def rank_range(rows: list[dict], world: int, rank: int) -> tuple[int, int]:
    """This rank's road range of a batch table (work = N x T per road)."""
    return road_ranges([int(r["N"]) * int(r["T"]) for r in rows], world)[rank]


def request_share(n_requests: int, world: int, rank: int) -> list[int]:
    """Arrival indices of the requests rank `rank` serves: every world-th."""
    if not (world >= 1 and 0 <= rank < world):
        raise ValueError("need world >= 1 and 0 <= rank < world")
    return list(range(rank, n_requests, world))
