"""tn_amplitudes_static: the entry point for callers that must not allocate device memory.

A caller whose memory pool already owns the GPU's memory, a host with a fixed memory budget, or
code running inside an allocator callback cannot let the library allocate. For them
tn_amplitudes_static computes the same amplitudes as tn_amplitudes from a fixed static scratch
array. These tests call it through the C ABI twice in a row and compare its results with those
of tn_amplitudes on the same plan, within the tolerances of the other GPU tests; they also check
that the PyTorch allocator the library is wired to sees no allocation during the calls, and that a
plan too large for the scratch is refused. This file is collected last on purpose."""
import numpy as np
import pytest

import gen
from tests.gpu_common import FP64_TOL, TC_TOL, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2011_02621_gb300 import build
    build.build()
    from paper_2011_02621_gb300 import tn as _tn
    return _tn


def _plan(tn, w, **opts):
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff)
    return tn.tn_path(c, **opts)


@pytest.mark.parametrize("name,n_bits,prec,tol", [
    ("grid12", 256, "fp64", FP64_TOL),
    ("grid12", 256, "fp32", TC_TOL),
    ("syc53", 48, "fp64", FP64_TOL),
    ("syc53", 48, "bf16x6", TC_TOL),
])
def test_static_matches_allocating_entry_point_twice(tn, name, n_bits, prec, tol):
    import torch
    w = gen.workload(name, n_bits=n_bits)
    p = _plan(tn, w)
    ref = tn.tn_amplitudes(p, w.bits, prec)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    a1 = tn.tn_amplitudes_static(p, w.bits, prec)
    a2 = tn.tn_amplitudes_static(p, w.bits, prec)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before       # nothing came from the allocator
    assert rel_err(a1, ref) < tol
    assert rel_err(a2, ref) < tol
    # results into a device tensor as well
    out = torch.zeros(len(w.bits), dtype=torch.complex128, device="cuda")
    tn.tn_amplitudes_static(p, w.bits, prec, out=out)
    assert rel_err(out.cpu().numpy(), ref) < tol


def test_static_rejects_plan_beyond_its_scratch(tn):
    """A 20-qubit, 14-cycle plan whose single slice needs about 100 MB is refused, not run."""
    w = gen.workload("grid20", n_bits=1)
    p = _plan(tn, w, max_intermediate=1 << 22)
    with pytest.raises(tn.TNError) as ei:
        tn.tn_amplitudes_static(p, w.bits, "bf16x6")
    assert ei.value.status == tn.TN_ERR_UNSUPPORTED
    assert "static scratch" in str(ei.value)


SCRATCH = 32 * 2 ** 20


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", TC_TOL)])
def test_static_runs_several_batches(tn, prec, tol):
    """More bitstrings than the scratch holds at once: the call runs them in several batches."""
    import torch
    w = gen.workload("syc53", n_bits=120)
    p = _plan(tn, w, layers=2)
    per = p.info["workspace_bytes"] / p.info["chunk_bitstrings"]       # one bitstring's workspace
    assert per * len(w.bits) > 2 * SCRATCH                             # at least three batches
    ref = tn.tn_amplitudes(p, w.bits, prec)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    for _ in range(2):
        assert rel_err(tn.tn_amplitudes_static(p, w.bits, prec), ref) < tol
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", TC_TOL)])
def test_static_splits_one_bitstring_into_slice_groups(tn, prec, tol):
    """A plan with 262144 slices whose single bitstring needs 128 MiB of workspace, more than the
    scratch, while one slice fits: each bitstring runs as several groups of its slices."""
    import torch
    w = gen.workload("grid12", n_bits=3)
    p = _plan(tn, w, max_intermediate=32)
    per = p.info["workspace_bytes"] / p.info["chunk_bitstrings"]
    assert p.info["n_slices"] >= 1 << 16 and per > SCRATCH
    ref = tn.tn_amplitudes(p, w.bits, prec)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    for _ in range(2):
        assert rel_err(tn.tn_amplitudes_static(p, w.bits, prec), ref) < tol
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
