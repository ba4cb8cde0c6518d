"""Sharding amplitude work over ranks (one process per GPU).

Bitstrings are independent units of the method: every rank evolves the same ket (deterministic)
and takes a contiguous block of the bitstrings, and nothing is exchanged (weak scaling). When a
job has fewer bitstrings than ranks, the ranks share the slices of each bitstring instead: the
amplitude is the sum of the cut network's slices (cutting, overlap paragraph), so each rank sums a
contiguous block of slices and the per-rank partial sums are combined by one FP64 reduce in fixed
rank order on the host. The reduce goes through a host (gloo) process group of complex128 numbers,
never through the device data path.

The compute callback is what a rank runs on its share: ``compute(bits_block, slice_begin,
slice_end)`` returns complex128 partial sums over the slices [slice_begin, slice_end) for each row
of ``bits_block`` (on a GPU: ``tn_amplitudes_slices``)."""
from __future__ import annotations

from typing import Callable, Optional, Tuple

import numpy as np


def block(total: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous block [lo, hi) of ``total`` units for ``rank``; sizes differ by at most one."""
    if world <= 0 or not 0 <= rank < world or total < 0:
        raise ValueError(f"bad block request total={total} rank={rank} world={world}")
    q, r = divmod(total, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def assignment(n_bits: int, n_slices: int, rank: int, world: int) -> dict:
    """What ``rank`` computes: a block of the bitstrings with all slices when there are at least
    as many bitstrings as ranks, else all bitstrings with a block of the slices."""
    if n_bits >= world or n_slices <= 1:
        return {"mode": "bitstrings", "bits": block(n_bits, rank, world), "slices": (0, n_slices)}
    return {"mode": "slices", "bits": (0, n_bits), "slices": block(n_slices, rank, world)}


def reduce_fixed_order(partial: np.ndarray, group=None, dst: int = 0) -> Optional[np.ndarray]:
    """Sum of every rank's ``partial`` (complex128) on rank ``dst``, added in rank order 0, 1, ...
    in FP64 (the same bits whatever the arrival order); None on the other ranks."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    t = torch.from_numpy(np.ascontiguousarray(partial, dtype=np.complex128).view(np.float64).copy())
    parts = [torch.empty_like(t) for _ in range(world)] if rank == dst else None
    dist.gather(t, gather_list=parts, dst=dst, group=group)
    if rank != dst:
        return None
    total = np.zeros_like(np.asarray(partial, dtype=np.complex128))
    for p in parts:                       # fixed order
        total = total + p.numpy().view(np.complex128)
    return total


def gather_blocks(local: np.ndarray, n_total: int, group=None, dst: int = 0) -> Optional[np.ndarray]:
    """Concatenation, in rank order, of every rank's block of results (complex128) on ``dst``;
    block sizes follow :func:`block`. None on the other ranks."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    size = max(block(n_total, r, world)[1] - block(n_total, r, world)[0] for r in range(world))
    buf = np.zeros(size, dtype=np.complex128)
    buf[: len(local)] = local
    t = torch.from_numpy(buf.view(np.float64).copy())
    parts = [torch.empty_like(t) for _ in range(world)] if rank == dst else None
    dist.gather(t, gather_list=parts, dst=dst, group=group)
    if rank != dst:
        return None
    out = []
    for r, p in enumerate(parts):
        lo, hi = block(n_total, r, world)
        out.append(p.numpy().view(np.complex128)[: hi - lo])
    return np.concatenate(out)


def sharded_amplitudes(compute: Callable[[np.ndarray, int, int], np.ndarray], bits: np.ndarray, n_slices: int,
                       group=None, dst: int = 0) -> Optional[np.ndarray]:
    """Amplitudes of every row of ``bits`` on rank ``dst`` (None elsewhere), the work shared over
    the group's ranks by :func:`assignment`."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    a = assignment(len(bits), n_slices, rank, world)
    lo, hi = a["bits"]
    s0, s1 = a["slices"]
    local = np.asarray(compute(bits[lo:hi], s0, s1), dtype=np.complex128)
    if a["mode"] == "bitstrings":
        return gather_blocks(local, len(bits), group, dst)
    return reduce_fixed_order(local, group, dst)
