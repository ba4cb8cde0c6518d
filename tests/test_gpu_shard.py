"""tn_amplitudes_slices, the per-rank work when slices are sharded: partial sums over the blocks
of a partition of the slices add up, in FP64, to the amplitudes (the amplitude is the sum over the
cut indices). Ranks are emulated one after another on one GPU."""
import numpy as np
import pytest

import gen
from paper_2011_02621_gb300 import shard
from tests.gpu_common import FP64_TOL, TC_TOL, rel_err, statevector_amplitudes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2011_02621_gb300 import build
    build.build()
    from paper_2011_02621_gb300 import tn as _tn
    return _tn


@pytest.fixture(scope="module")
def grid20(tn):
    w = gen.workload("grid20", n_bits=2)
    c = tn.tn_build(20, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split)
    p = tn.tn_path(c, max_intermediate=1 << 22)
    assert p.info["n_slices"] >= 8
    return w, c, p


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("bf16x6", TC_TOL)])
def test_slice_blocks_sum_to_amplitudes(tn, grid20, prec, tol):
    w, c, p = grid20
    S = p.info["n_slices"]
    full = tn.tn_amplitudes(p, w.bits, prec)
    for world in (2, 3):
        total = np.zeros(len(w.bits), dtype=np.complex128)
        for r in range(world):                       # fixed rank order
            a = shard.assignment(1, S, r, world)
            assert a["mode"] == "slices"
            s0, s1 = a["slices"]
            total = total + tn.tn_amplitudes_slices(p, w.bits, prec, s0, s1)
        assert rel_err(total, full) < 1e-12
    ref = statevector_amplitudes(20, w.gates, w.bits)
    assert rel_err(full, ref) < tol


def test_slice_range_edges(tn, grid20):
    w, c, p = grid20
    S = p.info["n_slices"]
    assert np.all(tn.tn_amplitudes_slices(p, w.bits, "fp64", 5, 5) == 0)
    one = [tn.tn_amplitudes_slices(p, w.bits, "fp64", s, s + 1) for s in range(S)]
    assert rel_err(np.sum(one, axis=0), tn.tn_amplitudes(p, w.bits, "fp64")) < 1e-12
    for lo, hi in ((-1, 2), (3, 2), (0, S + 1)):
        with pytest.raises(tn.TNError) as ei:
            tn.tn_amplitudes_slices(p, w.bits, "fp64", lo, hi)
        assert ei.value.status == tn.TN_ERR_ARG
