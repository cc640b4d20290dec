"""Placement of independent simulations over ranks (one process per GPU).

Simulations never exchange data, so more GPUs serve more requests with no collective on
the data path: every rank computes the same deterministic assignment from the request
list and serves only its share.  The assignment balances the work (node updates, with
FP64 requests weighted by the FP64/FP32 cost ratio) greedily, largest first.
"""
from __future__ import annotations

FP64_COST = 18.0   # measured step-time ratio of the FP64 to the mixed form


def cost(req) -> float:
    work = float(req.side) * float(req.side) * float(req.steps)
    return work * (FP64_COST if req.precision == "fp64" else 1.0)


def assign(requests, world_size: int) -> list[int]:
    """Rank of every request (same order as `requests`), identical on every rank."""
    load = [0.0] * world_size
    ranks = [0] * len(requests)
    order = sorted(range(len(requests)), key=lambda k: (-cost(requests[k]), requests[k].rid))
    for k in order:
        r = min(range(world_size), key=lambda q: (load[q], q))
        ranks[k] = r
        load[r] += cost(requests[k])
    return ranks


def my_share(requests, rank: int, world_size: int) -> list:
    ranks = assign(requests, world_size)
    return [req for req, r in zip(requests, ranks) if r == rank]
