"""Sharding of independent registration problems over ranks (one GPU each).

A batch of problems has no exchange step: each rank registers its share with
one batched call on its own GPU and the 92-byte results are gathered on the
host.  There is no data-path collective; torch.distributed carries only the
results and the timing (max over ranks).

Problems are assigned by longest-processing-time-first over an estimated
cost, which every rank computes identically, so the partition needs no
communication.
"""
from __future__ import annotations

import numpy as np


def problem_cost(n: int, k1: int, k2: int = 2) -> float:
    """Relative cost of one registration: the upper-triangle SC^2 GEMM
    (n_pad^3 / 2), the pairwise compatibility test (n^2 / 2) and the K1 K2 x n
    verification, in units of one dense multiply-add (weights chosen from the
    measured stage times at n = 5000: GEMM ~ 1/3, compatibility ~ 1/7,
    verification ~ 1/9 of a registration)."""
    n_pad = (n + 255) // 256 * 256
    return n_pad ** 3 / 2.0 / 4.5e3 + n * n / 2.0 + 2.2 * k1 * k2 * n


def partition(costs, world: int):
    """Indices of the problems of each rank: longest-processing-time-first on
    `costs` (ties by index), each rank's list in ascending index order."""
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def gather_results(local, parts, rank, world, group=None):
    """Reassemble per-rank result lists (in each rank's `parts[rank]` order)
    into one list in problem order, on every rank."""
    import torch.distributed as dist
    allr = [None] * world
    dist.all_gather_object(allr, (rank, local), group=group)
    out = [None] * sum(len(p) for p in parts)
    for r, lst in allr:
        for i, res in zip(parts[r], lst):
            out[i] = res
    return out


def register_sharded(ctx, xs, ys, offsets, params, rank, world, group=None):
    """Register this rank's share of a batch (host arrays; `params` one per
    problem) and return every problem's result, in order, on every rank."""
    offsets = np.asarray(offsets, dtype=np.int64)
    num = offsets.shape[0] - 1
    costs = [problem_cost(int(offsets[b + 1] - offsets[b]), int(params[b].k1), int(params[b].k2))
             for b in range(num)]
    parts = partition(costs, world)
    mine = parts[rank]
    if mine:
        xm = np.concatenate([xs[offsets[b]:offsets[b + 1]] for b in mine])
        ym = np.concatenate([ys[offsets[b]:offsets[b + 1]] for b in mine])
        om = np.cumsum([0] + [int(offsets[b + 1] - offsets[b]) for b in mine]).astype(np.int64)
        local = ctx.register_batched(xm, ym, om, [params[b] for b in mine])
    else:
        local = []
    return gather_results(local, parts, rank, world, group)
