"""Data-parallel sharding of retarget jobs over GPUs (one process per GPU).

Clips are independent, so the units split across ranks with no exchange on
the data path.  Each rank carves its own share with its own handle or
server.  The partition is a pure function of the job list and the world size,
so every rank computes the same one without communicating.  Longest
processing time first: jobs sorted by estimated cost (ties by index) go
one by one to the least-loaded rank (ties to the lowest rank).
"""
from __future__ import annotations


def job_cost(T: int, H: int, W: int, target_W: int, target_H: int, k: int) -> float:
    """Estimated work of a job.  Each pass scans T*H*W pixels once and then
    runs about ceil(removed / k) iterations over T*H*W-sized buffers."""
    cost = 0.0
    Wc = W
    if target_W < W:
        cost += T * H * W * (1.0 + (W - target_W) / max(k, 1))
        Wc = target_W
    if target_H < H:
        cost += T * H * Wc * (1.0 + (H - target_H) / max(k, 1))
    return cost


def partition(costs: list[float], world: int) -> list[int]:
    """Rank of every job (a list as long as costs)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    owner = [0] * len(costs)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += costs[i]
    return owner


def my_jobs(specs: list[dict], rank: int, world: int) -> list[int]:
    """Indices of the jobs this rank carves.  specs are dicts with T, H, W,
    target_W, target_H and k."""
    costs = [job_cost(s["T"], s["H"], s["W"], s["target_W"], s["target_H"], s["k"])
             for s in specs]
    owner = partition(costs, world)
    return [i for i, o in enumerate(owner) if o == rank]
