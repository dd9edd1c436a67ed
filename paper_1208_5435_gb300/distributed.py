"""Solving one caller's batch on several GPUs (one process per GPU, torch.distributed).

The problems of a batch are independent, so they shard without any exchange on the data
path: every rank receives the whole (host-side) description of the batch, takes the share
that a cost-balanced partition assigns it, solves that share with ONE mfipm_solve_batched
on its own GPU, and the solutions and infos are gathered once at the end.  A single
problem does not shard (its FFT would need an all-to-all per operator product and an
all-reduce per PCG iteration); it is solved by the rank it is assigned to.

Cost model: a partial-DCT problem costs ~ n log2 n per operator product and a dense one
~ m n; the iteration counts are about the same for every problem of a batch (the IPM takes
10-20 iterations, Sec. 5.1), so the partition balances n log2 n (resp. m n) by the LPT rule:
problems in decreasing cost, each to the rank with the least work so far.
"""
from __future__ import annotations

import heapq
import math
from typing import Callable, List, Optional, Sequence


def problem_cost(n: int, m: int, kind: str = "dct") -> float:
    """Relative cost of one solve (per operator product): n log2 n for the FFT-based
    operators, m n for a dense A."""
    if kind == "dense":
        return float(m) * float(n)
    return float(n) * math.log2(max(n, 2))


def partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Longest-processing-time assignment of problem indices to `world` ranks: indices in
    decreasing cost (ties by index), each to the rank with the least total so far (ties to the
    lowest rank).  Deterministic, so every rank computes the same partition; each rank's list
    is ascending."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    shards: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(s) for s in shards]


def solve_sharded(ops: Sequence, bs: Sequence, taus: Sequence[float], params=None, group=None,
                  local_solve: Optional[Callable] = None, gather_to: Optional[int] = None):
    """Solve the batch (ops[i], bs[i], taus[i]) across the ranks of `group` (default: the
    world).  Every rank passes the same batch description; rank r solves partition(...)[r]
    on its current CUDA device in one persistent launch.  Returns (xs, infos) with xs[i] a
    float64 CPU tensor and infos[i] the problem's info dict, on every rank (gather_to=None)
    or on rank gather_to only (others get None).  `local_solve(ops, bs, taus, params)` replaces
    the GPU solve (it must return (xs, infos) like solve_batched); it exists so that the
    partition and gather logic can run without a GPU."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    kinds = ["dense" if getattr(o, "A", None) is not None and not hasattr(o, "rows") else "dct" for o in ops]
    costs = [problem_cost(o.n, o.m, k) for o, k in zip(ops, kinds)]
    shards = partition(costs, world)
    mine = shards[rank]
    if local_solve is None:
        from . import solve_batched as local_solve
    if mine:
        xs, infos = local_solve([ops[i] for i in mine], [bs[i] for i in mine], [taus[i] for i in mine], params)
        part = (mine, [x.detach().to("cpu") for x in xs], list(infos))
    else:
        part = ([], [], [])
    if world == 1:
        gathered = [part]
    elif gather_to is None:
        gathered = [None] * world
        dist.all_gather_object(gathered, part, group=group)
    else:
        gathered = [None] * world if rank == gather_to else None
        dist.gather_object(part, gathered, dst=gather_to, group=group)
        if rank != gather_to:
            return None, None
    xs_all: List = [None] * len(ops)
    infos_all: List = [None] * len(ops)
    for idx, xs, infos in gathered:
        for i, x, inf in zip(idx, xs, infos):
            xs_all[i] = x if isinstance(x, torch.Tensor) else torch.as_tensor(x)
            infos_all[i] = inf
    return xs_all, infos_all
