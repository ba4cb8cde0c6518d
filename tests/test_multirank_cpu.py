"""Sharding over ranks, on CPU with world-size-2 gloo groups (one process per rank).

The per-rank compute is the oracle, so these tests run without a GPU; they check the host logic
that a multi-GPU job uses: bitstring blocks cover every bitstring once and need no exchange but
the final gather, and with fewer bitstrings than ranks the slice blocks' partial sums, reduced in
fixed rank order in FP64, give the full amplitude (the sum over the cut indices)."""
import os
import socket
import tempfile

import numpy as np
import pytest

import gen
from oracle import tns as otns
from paper_2011_02621_gb300 import shard


def test_blocks_partition_every_range():
    for total in (0, 1, 2, 3, 7, 64, 65537):
        for world in (1, 2, 3, 4, 8):
            spans = [shard.block(total, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == total
            assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1


def test_assignment_modes():
    assert shard.assignment(65536, 1, 1, 2) == {"mode": "bitstrings", "bits": (32768, 65536), "slices": (0, 1)}
    assert shard.assignment(1, 64, 1, 2) == {"mode": "slices", "bits": (0, 1), "slices": (32, 64)}
    assert shard.assignment(1, 1, 1, 2)["mode"] == "bitstrings"      # nothing to split: rank 1 idles
    with pytest.raises(ValueError):
        shard.block(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir, case):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        w = gen.workload("grid12", n_bits=case["n_bits"])
        cuts = case["cuts"]
        g1, g2 = otns.split_gates(w.gates, w.split)
        ket = otns.evolve_ket(w.graph.n, w.graph.edges, g1)

        def compute(bits, s0, s1):
            out, _ = otns.amplitudes(w.graph.n, w.graph.edges, w.gates, bits, w.split, cuts=cuts, ket=ket,
                                     slices=range(s0, s1))
            return out

        n_slices = 1
        if cuts:
            bra = otns.evolve_bra(w.graph.n, w.graph.edges, g2, w.bits[0])
            for e in cuts:
                n_slices *= ket.bond(e) * bra.bond(e)
        res = shard.sharded_amplitudes(compute, w.bits, n_slices)
        if rank == 0:
            np.save(os.path.join(out_dir, "result.npy"), res)
            np.save(os.path.join(out_dir, "n_slices.npy"), np.array([n_slices]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run_two_ranks(case):
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(2, _free_port(), d, case), nprocs=2, start_method="spawn", join=True)
        return np.load(os.path.join(d, "result.npy")), int(np.load(os.path.join(d, "n_slices.npy"))[0])


def test_two_ranks_bitstring_blocks_gloo():
    res, _ = _run_two_ranks({"n_bits": 9, "cuts": []})
    w = gen.workload("grid12", n_bits=9)
    ref, _ = otns.amplitudes(w.graph.n, w.graph.edges, w.gates, w.bits, w.split)
    assert res.shape == (9,)
    assert np.array_equal(res, ref)         # the same computation per bitstring, only moved


def test_two_ranks_slice_blocks_gloo():
    """One bitstring, two cut edges: rank 0 sums the first half of the slices, rank 1 the rest,
    and the fixed-order FP64 reduce gives the uncut amplitude."""
    res, n_slices = _run_two_ranks({"n_bits": 1, "cuts": [3, 10]})
    assert n_slices > 2
    w = gen.workload("grid12", n_bits=1)
    ref, _ = otns.amplitudes(w.graph.n, w.graph.edges, w.gates, w.bits, w.split)
    assert abs(res[0] - ref[0]) <= 1e-13 * max(abs(ref[0]), 1e-3)
