"""Contraction-path scores (oracle; test infrastructure only).

The supplement defines a sequential contraction path as an ordered qubit list
(Eq. path), the intermediate C^{i_1..i_m} of a set of qubits, and the score
S_{i_1..i_m i_{m+1}} = S_{i_1..i_m} + Cost(C^{i_1..i_m}, C^{i_{m+1}}) with
S_{i_1} = 0 (score recursion of the supplement). The optimum over all orders
satisfies the subset recursion Eq. optscore.

Cost(A, B) is not spelled out in the paper ("the computational complexity of
contracting" A and B). Reading used here: the number of complex
multiply-adds of the pairwise contraction, i.e. the product of the
dimensions of every leg of either tensor (shared legs counted once).

Two independent evaluations of the unconstrained optimum:

* ``bruteforce_optimum``: minimum of the score over all N! orders.
* ``subset_dp_optimum``: Eq. optscore as a dynamic programme over subsets.
"""
from __future__ import annotations

import itertools
from typing import List, Sequence, Tuple


def open_legs(mask: int, edges: Sequence[Tuple[int, int]]) -> List[int]:
    """Edges with exactly one endpoint in the set ``mask`` (legs of C^S)."""
    return [e for e, (u, v) in enumerate(edges) if ((mask >> u) & 1) != ((mask >> v) & 1)]


def cost(mask: int, i: int, edges, dims) -> int:
    """Cost(C^S, C^i): product of the dims of the union of the legs of C^S and C^i."""
    legs = set(open_legs(mask, edges))
    legs.update(e for e, (u, v) in enumerate(edges) if i in (u, v))
    c = 1
    for e in legs:
        c *= int(dims[e])
    return c


def score(order: Sequence[int], edges, dims) -> int:
    """S of a full or partial path (S = 0 for a single qubit)."""
    s = 0
    mask = 0
    for k, i in enumerate(order):
        if k > 0:
            s += cost(mask, i, edges, dims)
        mask |= 1 << i
    return s


def bruteforce_optimum(n: int, edges, dims) -> int:
    return min(score(p, edges, dims) for p in itertools.permutations(range(n)))


def subset_dp_optimum(n: int, edges, dims) -> int:
    """Eq. optscore: opt(S) = min_{i in S} opt(S minus i) + Cost(C^{S minus i}, C^i)."""
    full = (1 << n) - 1
    INF = float("inf")
    opt = [INF] * (full + 1)
    for i in range(n):
        opt[1 << i] = 0
    for mask in range(1, full + 1):
        if mask & (mask - 1) == 0:
            continue
        best = INF
        m = mask
        while m:
            low = m & -m
            i = low.bit_length() - 1
            rest = mask ^ low
            c = opt[rest] + cost(rest, i, edges, dims)
            if c < best:
                best = c
            m ^= low
        opt[mask] = best
    return int(opt[full])
