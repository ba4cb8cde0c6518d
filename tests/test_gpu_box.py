"""The box-tiled streaming step kernel (SIMT, thin steps) on the device, through the C ABI.

Every step that the kernel supports (K * N <= 4096, N <= 256) is forced onto it, the others keep
the shape heuristic's kernels, and the amplitudes are compared element by element with what
does not depend on the CUDA path: the brute-force state vector (untruncated 3x4 and 4x5 grids)
and the oracle's own contraction of the double-layer network (the 53-qubit workload, truncated).
Plans with cuts run several (bitstring, slice) items per bitstring. Tolerances as in the other
GPU tests: 1e-10 relative to rms|a| in FP64, 1e-5 in complex64."""
import numpy as np
import pytest

import gen
from oracle import statevector as sv
from oracle import tns as otns
from tests.gpu_common import FP64_TOL, TC_TOL, rel_err

pytestmark = pytest.mark.gpu

BOX_MAXKN, BOX_MAXN = 4096, 256


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2011_02621_gb300 import build
    build.build()
    from paper_2011_02621_gb300 import tn as _tn
    return _tn


def force_box(tn, p, prec):
    """Put every supported step on the box kernel; returns how many steps that is."""
    _, _, steps = tn.tn_plan_details(p)
    ks = ["simt_box" if (k * n <= BOX_MAXKN and n <= BOX_MAXN) else "simt_auto" for m, k, n in steps]
    tn.tn_plan_set_kernels(p, prec, ks)
    assert tn.tn_plan_kernels(p, prec) == ks
    return ks.count("simt_box")


@pytest.mark.parametrize("layers", [1, 2])
@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", TC_TOL)])
def test_box_grid12_vs_statevector(tn, layers, prec, tol):
    w = gen.workload("grid12", n_bits=64)
    ref = sv.amplitudes(sv.run(12, w.gates), w.bits)
    c = tn.tn_build(12, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, 0, 1e-12)
    for merge in (False, True):
        p = tn.tn_path(c, layers=layers, merge=merge)
        assert force_box(tn, p, prec) >= (20 if layers == 2 and not merge else 1)
        assert rel_err(tn.tn_amplitudes(p, w.bits, prec), ref) < tol, merge


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", TC_TOL)])
def test_box_with_cuts_vs_statevector(tn, prec, tol):
    """Cut plans: each bitstring is several items (one per slice) and the tables offset the cut legs."""
    w = gen.workload("grid12", n_bits=16)
    ref = sv.amplitudes(sv.run(12, w.gates), w.bits)
    c = tn.tn_build(12, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, 0, 1e-12)
    for layers in (1, 2):
        p = tn.tn_path(c, layers=layers, max_intermediate=64)
        assert p.info["n_slices"] > 1
        force_box(tn, p, prec)
        assert rel_err(tn.tn_amplitudes(p, w.bits, prec), ref) < tol, layers


def test_box_grid20_double_layer_vs_statevector(tn):
    """The 4x5 grid at 14 cycles (the precision workload) on its double-layer plan, FP64 and FP32."""
    w = gen.workload("grid20", n_bits=32)
    ref = sv.amplitudes(sv.run(20, w.gates), w.bits)
    c = tn.tn_build(20, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, 0, 1e-12)
    p = tn.tn_path(c, layers=2)
    for prec, tol in (("fp64", FP64_TOL), ("fp32", TC_TOL)):
        force_box(tn, p, prec)
        assert rel_err(tn.tn_amplitudes(p, w.bits, prec), ref) < tol, prec


@pytest.fixture(scope="module")
def syc53_double_layer_oracle():
    """The oracle's amplitudes of 16 bitstrings of the 53-qubit workload, contracted as the
    double-layer network (every ket and bra tensor a node of its own) in the oracle's own order."""
    w = gen.workload("syc53", n_bits=16)
    g1, g2 = otns.split_gates(w.gates, w.split)
    ket = otns.evolve_ket(w.graph.n, w.graph.edges, g1, w.chi, w.cutoff)
    ref = np.array([otns.double_layer_amplitude(ket, otns.evolve_bra(w.graph.n, w.graph.edges, g2, b, w.chi, w.cutoff))
                    for b in w.bits])
    return w, ref


@pytest.mark.parametrize("merge", [False, True])
@pytest.mark.parametrize("mode", ["box", "autotuned"])
def test_syc53_double_layer_vs_oracle_double_layer(tn, syc53_double_layer_oracle, mode, merge):
    """merge=False: one step per ket or bra tensor (every step on the box kernel); merge=True (the
    default): consecutive tensors of one layer joined first (the pair contracted on its own, in FP64)."""
    w, ref = syc53_double_layer_oracle
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff)
    p = tn.tn_path(c, layers=2, merge=merge)
    assert (p.info["n_nodes"] == 2 * w.graph.n) == (not merge)
    for prec, tol in (("fp64", FP64_TOL), ("fp32", TC_TOL)):
        if mode == "box":
            nb = force_box(tn, p, prec)
            assert nb == p.info["n_steps"] if not merge else nb >= p.info["n_steps"] - 2
        else:
            tn.tn_autotune(p, prec, 256)
        assert rel_err(tn.tn_amplitudes(p, w.bits, prec), ref) < tol, prec


def test_box_large_batch_sampled_vs_oracle(tn, syc53_double_layer_oracle):
    """A full device batch (16384 bitstrings, the launch shape the benchmark times) with the
    oracle's 16 bitstrings placed at the start, the middle and the end of it."""
    w, ref = syc53_double_layer_oracle
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff)
    p = tn.tn_path(c, layers=2)
    force_box(tn, p, "fp32")
    B = 16384
    bits = gen.bitstrings(w.graph.n, B, gen.rng(7, 2))
    pos = np.concatenate([np.arange(6), B // 2 + np.arange(5), B - 5 + np.arange(5)])
    bits[pos] = w.bits
    a = tn.tn_amplitudes(p, bits, "fp32")
    assert rel_err(a[pos], ref) < TC_TOL
    assert np.all(np.isfinite(a))
