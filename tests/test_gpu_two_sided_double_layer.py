"""The two-sided bond compression and the double-layer network on the device, through the C ABI.

* Two-sided compression (the singular values of the local product of a gate's two endpoints,
  run as two gate-kernel entries per gate): a 3x4 grid with Haar-random gates, every gate in the
  ket, bonds capped at chi = 4, so both compressions truncate; each form's FP64 amplitudes
  against the oracle run with the same compression.
* Double-layer plans (ket and bra tensors as separate nodes, one absorbed per step with the unit
  operand): the 3x4 grid against its state vector, and the 53-qubit workload against the
  overlap network's FP64 amplitudes, in FP64 and FP32.

Tolerances as in the other GPU tests: 1e-10 relative to rms|a| in FP64, 1e-5 in complex64."""
import numpy as np
import pytest

import gen
from oracle import statevector as sv
from oracle import tns as otns
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


@pytest.mark.parametrize("compress", ["one_sided", "two_sided"])
def test_capped_haar_grid_matches_the_oracle_in_each_compression(tn, compress):
    g = gen.grid(3, 4)
    gates = gen.rqc(g, 8, gen.rng(44, 1), twoq="haar", oneq="haar")
    bits = gen.bitstrings(12, 16, gen.rng(44, 2))
    c = tn.tn_build(12, g.edges, gates)
    tn.tn_evolve_two_sided(c, 8, 4, 1e-12, compress=compress)
    a = tn.tn_amplitudes(tn.tn_path(c), bits, "fp64")
    ref, _ = otns.amplitudes(12, g.edges, gates, bits, 8, 4, 1e-12, compress=compress)
    assert rel_err(a, ref) < FP64_TOL


@pytest.mark.parametrize("merge", [False, True])
@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", TC_TOL)])
def test_double_layer_grid12_vs_statevector(tn, prec, tol, merge):
    """merge=False: one node per ket and per bra tensor; merge=True (default): consecutive
    tensors of one layer joined (contracted with each other first, in FP64) where that is cheaper."""
    w = gen.workload("grid12", n_bits=32)
    ref = sv.amplitudes(sv.run(12, w.gates), w.bits)
    c = tn.tn_build(12, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, 0, 1e-12)
    p = tn.tn_path(c, layers=2, merge=merge)
    assert (p.info["n_steps"] == 23) == (not merge)
    assert rel_err(tn.tn_amplitudes(p, w.bits, prec), ref) < tol


@pytest.mark.parametrize("merge", [False, True])
@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", TC_TOL)])
def test_double_layer_syc53_vs_overlap_network(tn, prec, tol, merge):
    w = gen.workload("syc53", n_bits=64)
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff)
    a64 = tn.tn_amplitudes(tn.tn_path(c), w.bits, "fp64")
    p = tn.tn_path(c, layers=2, merge=merge)
    assert (p.info["n_nodes"] == 2 * w.graph.n) == (not merge)
    assert rel_err(tn.tn_amplitudes(p, w.bits, prec), a64) < tol
