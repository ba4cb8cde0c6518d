"""Parity of the CUDA path (through the C ABI) with the CPU oracle and the
brute-force state vector, element by element, on seeded inputs.

Tolerances: |da|/rms|a| <= 1e-10 for the FP64 path and <= 1e-5 for the
complex64 paths (FP32 SIMT and the tensor-core forms)."""
import math

import numpy as np
import pytest

import gen
from tests.gpu_common import (FP64_TOL, TC_TOL, gpu_amplitudes, oracle_amplitudes, rel_err,
                              statevector_amplitudes)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2011_02621_gb300 import build
    build.build()
    from paper_2011_02621_gb300 import tn as _tn
    return _tn


def test_grid12_fp64_all_bitstrings_vs_statevector(tn):
    w = gen.workload("grid12")
    ref = statevector_amplitudes(12, w.gates, w.bits)
    a, _, p = gpu_amplitudes(tn, 12, w.graph.edges, w.gates, w.bits, w.split)
    assert rel_err(a, ref) < FP64_TOL
    assert tn.tn_launch_count() > 0


def test_grid12_every_split_fp64(tn):
    w = gen.workload("grid12", n_bits=64)
    ref = statevector_amplitudes(12, w.gates, w.bits)
    for split in range(0, w.depth + 1):
        a, _, _ = gpu_amplitudes(tn, 12, w.graph.edges, w.gates, w.bits, split)
        assert rel_err(a, ref) < FP64_TOL, split


def test_grid12_oracle_elementwise(tn):
    w = gen.workload("grid12", n_bits=64)
    ref = oracle_amplitudes(12, w.graph.edges, w.gates, w.bits, w.split)
    a, _, _ = gpu_amplitudes(tn, 12, w.graph.edges, w.gates, w.bits, w.split)
    assert rel_err(a, ref) < FP64_TOL


def test_grid12_fp32(tn):
    w = gen.workload("grid12")
    ref = statevector_amplitudes(12, w.gates, w.bits)
    a, _, _ = gpu_amplitudes(tn, 12, w.graph.edges, w.gates, w.bits, w.split, prec="fp32")
    assert rel_err(a, ref) < TC_TOL


def test_structural_bonds_bound_oracle_ranks(tn):
    """Bond shapes after the rank probe: the ket's equal the oracle's true ranks at every split,
    the bra's bound the true ranks of every bitstring (Eqs. svd, shouwei); on the 53-qubit
    workload both are exact."""
    from oracle import tns as otns
    w = gen.workload("grid12", n_bits=4)
    c = tn.tn_build(12, w.graph.edges, w.gates)
    for split in (2, 4, 6):
        tn.tn_evolve_two_sided(c, split, 0, 1e-12)
        g1, g2 = otns.split_gates(w.gates, split)
        ket = otns.evolve_ket(12, w.graph.edges, g1)
        assert list(tn.tn_circuit_bond_dims(c, 0)) == ket.bonds()
        sb = tn.tn_circuit_bond_dims(c, 1)
        for b in w.bits:
            bra = otns.evolve_bra(12, w.graph.edges, g2, b)
            assert all(int(x) >= y for x, y in zip(sb, bra.bonds()))
    w = gen.workload("syc53", n_bits=3)
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff)
    g1, g2 = otns.split_gates(w.gates, w.split)
    assert list(tn.tn_circuit_bond_dims(c, 0)) == otns.evolve_ket(w.graph.n, w.graph.edges, g1, w.chi, w.cutoff).bonds()
    for b in w.bits:
        bra = otns.evolve_bra(w.graph.n, w.graph.edges, g2, b, w.chi, w.cutoff)
        assert list(tn.tn_circuit_bond_dims(c, 1)) == bra.bonds()


def test_cuts_give_same_amplitudes(tn):
    w = gen.workload("grid12", n_bits=48)
    ref = statevector_amplitudes(12, w.gates, w.bits)
    for cuts in ([3], [0, 7], [5, 9, 12]):
        a, _, p = gpu_amplitudes(tn, 12, w.graph.edges, w.gates, w.bits, w.split, cut_edges=cuts)
        assert p.info["n_cuts"] == len(cuts) and p.info["n_slices"] > 1
        assert rel_err(a, ref) < FP64_TOL, cuts
    a, _, p = gpu_amplitudes(tn, 12, w.graph.edges, w.gates, w.bits, w.split, max_intermediate=64)
    assert p.info["n_cuts"] > 0 and p.info["max_intermediate"] <= 64 * 16
    assert rel_err(a, ref) < FP64_TOL


def test_random_regular_haar_graphs(tn):
    for i, n in enumerate((10, 14, 16)):
        g = gen.random_regular3(n, gen.rng(300 + i, 0))
        gates = gen.rqc(g, 6, gen.rng(300 + i, 1), sequence="".join(sorted(g.patterns)), oneq="haar")
        bits = gen.bitstrings(n, 40, gen.rng(300 + i, 2))
        ref = statevector_amplitudes(n, gates, bits)
        a, _, _ = gpu_amplitudes(tn, n, g.edges, gates, bits, 3)
        assert rel_err(a, ref) < FP64_TOL


def test_general_two_qubit_gates(tn):
    g = gen.grid(3, 3)
    gates = gen.rqc(g, 6, gen.rng(41, 1), twoq="haar")
    bits = gen.bitstrings(9, 64, gen.rng(41, 2))
    ref = statevector_amplitudes(9, gates, bits)
    for split in (0, 3, 6):
        a, _, _ = gpu_amplitudes(tn, 9, g.edges, gates, bits, split)
        assert rel_err(a, ref) < FP64_TOL


def test_graph_state_closed_form_53_and_104(tn):
    for g in (gen.staggered(6, 9, remove_seed=gen.BASE_SEED + 3), gen.staggered(8, 13)):
        gates = gen.graph_state_circuit(g)
        bits = gen.bitstrings(g.n, 256, gen.rng(6, 2))
        par = np.array([sum(int(b[u]) * int(b[v]) for u, v in g.edges) for b in bits])
        expect = 2.0 ** (-g.n / 2) * (-1.0) ** par
        for split in (0, 1):
            a, _, _ = gpu_amplitudes(tn, g.n, g.edges, gates, bits, split)
            assert rel_err(a, expect) < FP64_TOL


def test_mirror_circuit_delta(tn):
    """U then U^dagger with the split between them: a(s) = delta_{s,0}; the bra half is U^dagger."""
    g = gen.grid(3, 4)
    gates = gen.mirror_circuit(gen.rqc(g, 4, gen.rng(3, 1)))
    bits = np.vstack([np.zeros(12, np.uint8), gen.bitstrings(12, 15, gen.rng(3, 2))])
    a, _, _ = gpu_amplitudes(tn, 12, g.edges, gates, bits, 4)
    assert abs(a[0] - 1) < 1e-10 and np.max(np.abs(a[1:])) < 1e-10


def test_slice_groups_when_one_bitstring_exceeds_budget(tn):
    """Slices of one bitstring processed in groups, summed in order in FP64, equal the unsliced result."""
    w = gen.workload("grid12", n_bits=6)
    ref = statevector_amplitudes(12, w.gates, w.bits)
    c = tn.tn_build(12, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split)
    info = tn.tn_path(c, cut_edges=[0, 7]).info
    S, maxT = info["n_slices"], info["max_intermediate"]
    assert S >= 4
    budget = (S // 3) * 2 * maxT * 16 + 2 ** 20        # about a third of one bitstring's slices fits
    p = tn.tn_path(c, cut_edges=[0, 7], mem_budget_bytes=budget)
    assert p.info["chunk_bitstrings"] == 1
    assert rel_err(tn.tn_amplitudes(p, w.bits), ref) < FP64_TOL


def test_syc53_truncated_vs_oracle(tn):
    """53 qubits, 10 cycles, split 5, chi 64, cutoff 1e-8: sampled bitstrings vs the step-by-step oracle."""
    w = gen.workload("syc53", n_bits=32)
    ref = oracle_amplitudes(w.graph.n, w.graph.edges, w.gates, w.bits, w.split, w.chi, w.cutoff)
    a, _, _ = gpu_amplitudes(tn, w.graph.n, w.graph.edges, w.gates, w.bits, w.split, w.chi, w.cutoff)
    assert rel_err(a, ref) < FP64_TOL
    a32, _, _ = gpu_amplitudes(tn, w.graph.n, w.graph.edges, w.gates, w.bits, w.split, w.chi, w.cutoff,
                               prec="fp32")
    assert rel_err(a32, ref) < TC_TOL


def test_edge_cases(tn):
    # empty batch
    w = gen.workload("grid12", n_bits=4)
    c = tn.tn_build(12, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split)
    p = tn.tn_path(c)
    assert tn.tn_amplitudes(p, np.zeros((0, 12), np.uint8)).shape == (0,)
    # one bitstring, ragged chunk (budget forces chunks of a few bitstrings)
    ref = statevector_amplitudes(12, w.gates, w.bits)
    p2 = tn.tn_path(c, mem_budget_bytes=1)
    assert p2.info["chunk_bitstrings"] == 1
    assert rel_err(tn.tn_amplitudes(p2, w.bits), ref) < FP64_TOL
    assert rel_err(tn.tn_amplitudes(p, w.bits[:1]), ref[:1]) < FP64_TOL
    # two qubits, one edge; one qubit, no edges
    g = gen.grid(1, 2)
    gates = gen.rqc(g, 3, gen.rng(2, 1))
    bits = gen.all_bitstrings(2)
    a, _, _ = gpu_amplitudes(tn, 2, g.edges, gates, bits, 1)
    assert rel_err(a, statevector_amplitudes(2, gates, bits)) < FP64_TOL
    one = [gen.Gate(1, (0,), gen.SQRT_X), gen.Gate(2, (0,), gen.SQRT_Y)]
    a, _, _ = gpu_amplitudes(tn, 1, [], one, gen.all_bitstrings(1), 1)
    assert rel_err(a, statevector_amplitudes(1, one, gen.all_bitstrings(1))) < FP64_TOL


def test_device_buffers_in_and_out(tn):
    import torch
    w = gen.workload("grid12", n_bits=100)
    ref = statevector_amplitudes(12, w.gates, w.bits)
    c = tn.tn_build(12, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split)
    p = tn.tn_path(c)
    bits_dev = torch.from_numpy(tn.pack_bits(w.bits).view(np.int64)).cuda()
    out = torch.zeros(100, dtype=torch.complex128, device="cuda")
    tn.tn_amplitudes(p, bits_dev, "fp64", out=out)
    assert rel_err(out.cpu().numpy(), ref) < FP64_TOL


# per-form bound on |da|/rms|a|: the six-product forms carry ~24-bit products and meet 1e-5;
# the two-piece forms (~21 and ~17 bits) are kept for comparison with looser bounds
TC_BOUND = {"bf16x6": TC_TOL, "tf32x6": 3e-5, "tf32x3": 5e-5, "bf16x3": 2e-4, "tf32": 2e-2}


@pytest.mark.parametrize("prec", ["bf16x6", "tf32x6", "tf32x3", "bf16x3"])
def test_tensor_core_grid12_vs_statevector(tn, prec):
    w = gen.workload("grid12")
    ref = statevector_amplitudes(12, w.gates, w.bits)
    a, _, _ = gpu_amplitudes(tn, 12, w.graph.edges, w.gates, w.bits, w.split, prec=prec)
    assert rel_err(a, ref) < TC_BOUND[prec]


def test_tensor_core_single_pass_tf32_is_coarse_but_close(tn):
    """Single-pass TF32 (10-bit mantissa) misses 1e-5 by far but stays within a few 1e-3."""
    w = gen.workload("grid12")
    ref = statevector_amplitudes(12, w.gates, w.bits)
    a, _, _ = gpu_amplitudes(tn, 12, w.graph.edges, w.gates, w.bits, w.split, prec="tf32")
    assert rel_err(a, ref) < 2e-2


def test_tensor_core_syc53_vs_oracle_and_fp64(tn):
    w = gen.workload("syc53", n_bits=48)
    ref = oracle_amplitudes(w.graph.n, w.graph.edges, w.gates, w.bits, w.split, w.chi, w.cutoff)
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff)
    p = tn.tn_path(c)
    a64 = tn.tn_amplitudes(p, w.bits, "fp64")
    assert rel_err(a64, ref) < FP64_TOL
    for prec in ("bf16x6", "tf32x6", "tf32x3", "bf16x3", "tf32"):
        tn.tn_profile_enable(True)
        a = tn.tn_amplitudes(p, w.bits, prec)
        prof = tn.tn_profile_read()
        tn.tn_profile_enable(False)
        tc = sum(v["launches"] for k, v in prof.items() if k.startswith("contract_step_tcgen05"))
        assert tc > 0, prec
        assert rel_err(a, ref) < TC_BOUND[prec], prec
        assert rel_err(a, a64) < TC_BOUND[prec], prec


def test_tensor_core_cuts_and_ragged_tiles(tn):
    """Slices, M not a multiple of 128 and N not a multiple of the tile on the tcgen05 paths, on
    the deep 14-cycle circuit: FP32 SIMT and BF16x6 within 1e-5 (the tensor-core path's tolerance;
    BF16x6 steps with K >= 256 run on 64-column tiles, 7 order-0 accumulators), TF32x6 within its
    form's bound (products of 21-bit pieces, accumulated in FP32 by the tensor core)."""
    w = gen.workload("grid20", n_bits=4)
    ref = statevector_amplitudes(20, w.gates, w.bits)
    c = tn.tn_build(20, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split)
    p = tn.tn_path(c, max_intermediate=1 << 22)
    assert p.info["n_slices"] > 1
    assert rel_err(tn.tn_amplitudes(p, w.bits, "fp32"), ref) < 1e-5
    for prec, bound in (("bf16x6", TC_TOL), ("tf32x6", 4e-5)):
        assert rel_err(tn.tn_amplitudes(p, w.bits, prec), ref) < bound, prec


@pytest.mark.parametrize("name,n_bits,opts", [
    ("syc53", 32, {}),
    ("grid20", 2, {"max_intermediate": 1 << 22}),
    ("grid12", 64, {"cut_edges": [3, 10]}),
])
def test_node_merging_is_exact(tn, name, n_bits, opts):
    """Merging boundary nodes into neighbours (exact contractions of the ket and bra node tensors)
    leaves the amplitudes unchanged: merged and unmerged plans agree in FP64 and in BF16x6."""
    w = gen.workload(name, n_bits=n_bits)
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff)
    pm = tn.tn_path(c, **opts)
    pu = tn.tn_path(c, merge=False, **opts)
    assert pu.info["n_nodes"] == w.graph.n
    assert pm.info["n_nodes"] < w.graph.n
    assert pm.info["n_steps"] == pm.info["n_nodes"] - 1
    order, cuts, steps = tn.tn_plan_details(pm)
    reps = [q for q in order if q >= 0]
    assert len(reps) == pm.info["n_nodes"] and len(set(reps)) == len(reps)
    if "cut_edges" in opts:
        assert sorted(cuts) == sorted(opts["cut_edges"])
    a_m = tn.tn_amplitudes(pm, w.bits, "fp64")
    a_u = tn.tn_amplitudes(pu, w.bits, "fp64")
    assert rel_err(a_m, a_u) < 1e-12
    if name != "grid12":
        assert rel_err(tn.tn_amplitudes(pm, w.bits, "bf16x6"), a_u) < TC_TOL
