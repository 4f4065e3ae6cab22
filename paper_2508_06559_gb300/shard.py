"""Sharding one deal's exact solve over several solvers (one per GPU).

The FGT roots of a round are independent (open hands; every root's reach is 1, section "CFR
Algorithm"), so a round's GT roots can be cut into ranges solved by different ranks; the one
exchange per round is the round's average root utilities, which the previous round's leaves
need (eq. passuputil): every rank contributes its range (zero elsewhere) and a sum over ranks
gives the whole vector, bit for bit.  This module holds the host logic only: the partition and
the backward sweep over rounds with a pluggable range solver and a pluggable sum over ranks
(torch.distributed's all_reduce on the GPU ranks; gloo on CPU ranks in the tests).
"""
from __future__ import annotations

import numpy as np


def partition_roots(sizes, n_parts: int):
    """Contiguous ranges (first, count) of GT roots, one per part, balancing the parts' total size:
    part p takes the roots whose prefix of sizes before them lies in [p, p + 1) * total / n_parts.
    Every root belongs to exactly one part; parts may be empty."""
    s = np.asarray(sizes, np.float64)
    n = len(s)
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    total = float(s.sum())
    if n == 0 or total <= 0:
        cuts = [min(n, (p * n + n_parts - 1) // n_parts) for p in range(n_parts)] + [n]
    else:
        before = np.concatenate([[0.0], np.cumsum(s)[:-1]])
        cuts = [int(np.searchsorted(before, p * total / n_parts, side="left")) for p in range(n_parts)] + [n]
        cuts[0] = 0
    return [(cuts[p], cuts[p + 1] - cuts[p]) for p in range(n_parts)]


def sharded_backward(rounds, sizes_of, solve_range, sum_over_ranks, rank: int, world: int, dtype=np.float32):
    """Solve rounds (ordered first..last, the last one final) backward with rank `rank` of `world`
    taking one contiguous range of every round's GT roots.

    sizes_of(round) -> per GT root sizes to balance;  solve_range(round, u_next, first, count) ->
    float32 average root utilities of every FGT root of the round (zero outside the range);
    sum_over_ranks(u) -> the elementwise sum over all ranks (an all-reduce).  Utilities are passed
    as `dtype` (float32: what the GPU solver exchanges).  Returns the list of every round's whole
    utility vector (same order as rounds)."""
    out = [None] * len(rounds)
    u_next = None
    for i in range(len(rounds) - 1, -1, -1):
        first, count = partition_roots(sizes_of(rounds[i]), world)[rank]
        u_local = np.asarray(solve_range(rounds[i], u_next, first, count), dtype)
        u = np.asarray(sum_over_ranks(u_local), dtype)
        out[i] = u
        u_next = u
    return out
