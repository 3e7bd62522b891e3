"""Sharding of independent density matrices over ranks (one GPU per rank).

A single density matrix is not split across GPUs; the instances of a batch are independent,
so a multi-GPU run gives each rank a share of them (no collective on the data path) and
reduces only timings. The share is balanced by the cost of an instance, which grows like
N^3 (every product of an n x n instance is n^2 (n+1) flops per split product): the longest
instances are placed first, each on the rank with the least work so far (the LPT rule of
Graham 1969), ties to the lower rank, so every rank computes the same partition without
communication.
"""
from __future__ import annotations

import heapq

__all__ = ["instance_cost", "lpt_partition", "rank_share", "reduce_max"]


def instance_cost(n: int) -> float:
    return float(n) ** 2 * (float(n) + 1.0)


def lpt_partition(costs, parts: int) -> list[list[int]]:
    """Indices of `costs` split into `parts` lists by longest-processing-time-first."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(parts)]
    out: list[list[int]] = [[] for _ in range(parts)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    for lst in out:
        lst.sort()
    return out


def rank_share(ns, rank: int, world: int) -> list[int]:
    """Instances (indices into ns) that `rank` of `world` computes."""
    return lpt_partition([instance_cost(n) for n in ns], world)[rank]


def reduce_max(value: float) -> float:
    """Maximum of `value` over the ranks of the default process group (itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
