"""Pins of the CPU oracle against facts that the paper and the mathematics fix.

None of these compare the oracle with itself: the state vector is pinned by an
entry-by-entry unitary and by hand-derived gate actions; the TNS method is
pinned by the state vector (the untruncated method is exact), by closed forms
(graph states at 53 and 104 qubits, mirror circuits), by the split, slice and
path independence the method must have, and by the bond bounds of the paper
(chi_o of Eq. gatesplit, Eq. shouwei)."""
import itertools
import math

import numpy as np
import pytest

import gen
from oracle import path as opath
from oracle import statevector as sv
from oracle import tns

RNG = np.random.default_rng(7)


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.sqrt(np.mean(np.abs(b) ** 2)))


def small_random_circuit(graph, depth, seed):
    return gen.rqc(graph, depth, gen.rng(seed, 1))


# ---------------------------------------------------------------- state vector
def test_statevector_matches_entrywise_unitary():
    for (R, C), d in [((1, 3), 4), ((2, 2), 5), ((2, 3), 3)]:
        g = gen.grid(R, C)
        gates = small_random_circuit(g, d, 11 + R * C)
        psi = sv.run(g.n, gates)
        U = sv.unitary_bruteforce(g.n, gates)
        col = U[:, 0]
        for idx in range(1 << g.n):
            bits = tuple((idx >> q) & 1 for q in range(g.n))
            assert abs(psi[bits] - col[idx]) < 1e-13


def test_fsim_on_basis_states_by_hand():
    # fSim(theta, phi): |00> -> |00>, |01> -> cos|01> - i sin|10>, |11> -> e^{-i phi}|11>
    th, ph = 0.3, 1.1
    m = gen.fsim(th, ph)
    g = gen.Gate(1, (0, 1), m)
    for s0, s1 in itertools.product((0, 1), repeat=2):
        psi = np.zeros((2, 2), complex)
        psi[s0, s1] = 1
        out = sv.apply_gate(psi, (0, 1), m)
        exp = np.zeros((2, 2), complex)
        if (s0, s1) == (0, 0):
            exp[0, 0] = 1
        elif (s0, s1) == (1, 1):
            exp[1, 1] = np.exp(-1j * ph)
        else:
            exp[s0, s1] = math.cos(th)
            exp[s1, s0] = -1j * math.sin(th)
        assert np.allclose(out, exp, atol=1e-15)
    # qubit order: gate on (1, 0) applies the same matrix with qubit 1 as the high bit
    psi = np.zeros((2, 2), complex)
    psi[0, 1] = 1                                  # s_0 = 0, s_1 = 1
    cnot_like = np.eye(4, dtype=complex)[[0, 1, 3, 2]]   # flips the low bit if the high bit is 1
    out = sv.apply_gate(psi, (1, 0), cnot_like)    # high bit = qubit 1 = 1 -> flip qubit 0
    assert abs(out[1, 1] - 1) < 1e-15


def test_graph_state_statevector_closed_form():
    g = gen.grid(3, 3)
    psi = sv.run(g.n, gen.graph_state_circuit(g))
    bits = gen.all_bitstrings(g.n)
    par = np.zeros(len(bits), dtype=np.int64)
    for (u, v) in g.edges:
        par += bits[:, u].astype(np.int64) * bits[:, v]
    expect = 2.0 ** (-g.n / 2) * (-1.0) ** par
    assert rel_err(sv.amplitudes(psi, bits), expect) < 1e-13


def test_porter_thomas_deep_circuit():
    w = gen.workload("grid20", n_bits=1)
    psi = sv.run(w.graph.n, w.gates)
    p = (2 ** w.graph.n) * np.abs(psi.ravel()) ** 2
    assert abs(p.mean() - 1.0) < 1e-10               # normalisation
    assert abs(np.mean(p ** 2) - 2.0) < 0.05          # Porter-Thomas second moment


# ---------------------------------------------------------------- gate split
@pytest.mark.parametrize("m,chi_o", [
    (gen.fsim(math.pi / 2, math.pi / 6), 4),
    (gen.fsim(math.pi / 2, 0.0), 4),      # iSWAP-like
    (gen.fsim(0.0, math.pi), 2),          # CZ (a controlled gate)
    (np.eye(4, dtype=complex), 1),
    (np.eye(4, dtype=complex)[[0, 2, 1, 3]], 4),   # SWAP
    (np.eye(4, dtype=complex)[[0, 1, 3, 2]], 2),   # CNOT
])
def test_gate_split_chi_o_and_reconstruction(m, chi_o):
    P, Q, c = tns.gate_split(m)
    assert c == chi_o
    rec = np.einsum("aks,bls->abkl", P, Q).reshape(4, 4)
    assert np.max(np.abs(rec - m)) < 1e-14


# ---------------------------------------------------------------- the method
def test_tns_equals_statevector_every_split():
    w = gen.workload("grid12")
    psi = sv.run(w.graph.n, w.gates)
    ref = sv.amplitudes(psi, w.bits)
    for c in range(0, w.depth + 1):
        bits = w.bits if c == w.split else w.bits[:16]
        a, _ = tns.amplitudes(w.graph.n, w.graph.edges, w.gates, bits, c)
        assert rel_err(a, ref[: len(bits)]) < 1e-12, c


def test_tns_random_graphs_equal_statevector():
    for i, n in enumerate((6, 8, 10)):
        g = gen.random_regular3(n, gen.rng(100 + i, 0))
        gates = gen.rqc(g, 5, gen.rng(100 + i, 1), sequence="".join(sorted(g.patterns)), oneq="haar")
        psi = sv.run(n, gates)
        bits = gen.bitstrings(n, 12, gen.rng(100 + i, 2))
        a, _ = tns.amplitudes(n, g.edges, gates, bits, 2)
        assert rel_err(a, sv.amplitudes(psi, bits)) < 1e-12


def test_tns_general_two_qubit_gates_equal_statevector():
    """Eqs. gatesplit-svd2 hold for any two-qubit gate, not only fSim."""
    g = gen.grid(3, 3)
    gates = gen.rqc(g, 6, gen.rng(31, 1), twoq="haar")
    psi = sv.run(g.n, gates)
    bits = gen.bitstrings(g.n, 16, gen.rng(31, 2))
    for split in (0, 3, 6):
        a, _ = tns.amplitudes(g.n, g.edges, gates, bits, split)
        assert rel_err(a, sv.amplitudes(psi, bits)) < 1e-12


def test_normalisation_over_all_bitstrings():
    g = gen.grid(2, 4)
    gates = small_random_circuit(g, 6, 5)
    bits = gen.all_bitstrings(g.n)
    a, _ = tns.amplitudes(g.n, g.edges, gates, bits, 3)
    assert abs(np.sum(np.abs(a) ** 2) - 1.0) < 1e-12


def test_slice_independence():
    w = gen.workload("grid12", n_bits=6)
    g1, g2 = tns.split_gates(w.gates, w.split)
    ket = tns.evolve_ket(w.graph.n, w.graph.edges, g1)
    for bits in w.bits:
        bra = tns.evolve_bra(w.graph.n, w.graph.edges, g2, bits)
        full = tns.overlap_amplitude(ket, bra)
        for cuts in ([3], [0, 7], [5, 9, 12]):
            assert abs(tns.overlap_amplitude(ket, bra, cuts) - full) < 1e-13 * max(1.0, abs(full)) + 1e-16


def test_contraction_order_independence():
    w = gen.workload("grid12", n_bits=3)
    g1, g2 = tns.split_gates(w.gates, w.split)
    ket = tns.evolve_ket(w.graph.n, w.graph.edges, g1)
    for bits in w.bits:
        bra = tns.evolve_bra(w.graph.n, w.graph.edges, g2, bits)
        C = [tns.overlap_node(ket.A[q], bra.A[q]) for q in range(w.graph.n)]
        ref = tns.contract_network(C, ket.legs)
        # sequential absorption in random connected orders, one tensordot at a time
        for seed in range(3):
            r = np.random.default_rng(seed)
            order = [int(r.integers(w.graph.n))]
            while len(order) < w.graph.n:
                front = sorted({v for (a, b) in w.graph.edges for (u, v) in ((a, b), (b, a))
                                if u in order and v not in order})
                order.append(front[int(r.integers(len(front)))])
            t, lab = C[order[0]], list(ket.legs[order[0]])
            for q in order[1:]:
                sh = [x for x in lab if x in ket.legs[q]]
                t = np.tensordot(t, C[q], axes=([lab.index(x) for x in sh], [ket.legs[q].index(x) for x in sh]))
                lab = [x for x in lab if x not in sh] + [x for x in ket.legs[q] if x not in sh]
            assert abs(complex(t) - ref) < 1e-14


def test_bra_transpose_equals_dagger():
    """<psi| = <s| U2 : the transposed gates on |s> give conj(U2^dagger |s>)."""
    g = gen.grid(2, 3)
    gates = small_random_circuit(g, 4, 21)
    g1, g2 = tns.split_gates(gates, 2)
    bits = np.array([1, 0, 1, 1, 0, 0], dtype=np.uint8)
    bra = tns.evolve_bra(g.n, g.edges, g2, bits)
    dense = tns.to_dense(bra)
    psi = np.zeros((2,) * g.n, complex)
    psi[tuple(bits)] = 1
    for gt in reversed(g2):                       # U2^dagger |s>
        psi = sv.apply_gate(psi, gt.qubits, gt.m.conj().T)
    assert np.max(np.abs(dense - psi.conj())) < 1e-14


def test_first_application_bond_at_most_two():
    """Eq. shouwei: the first chi_o = 4 gate on a qubit leaves its bond <= 2."""
    w = gen.workload("grid12")
    g1 = [gt for gt in w.gates if gt.cycle == 1]
    ket = tns.evolve_ket(w.graph.n, w.graph.edges, g1)
    for e in w.graph.patterns["A"]:
        assert ket.bond(e) == 2
    assert all(b <= 2 for b in ket.bonds())


def test_bond_bounds_every_compression():
    """dim(s') <= min(dim(a) chi_o, 2 prod(other legs)) for every compression (Eqs. svd, shouwei)."""
    w = gen.workload("grid12")
    g1, g2 = tns.split_gates(w.gates, 6)
    ket = tns.evolve_ket(w.graph.n, w.graph.edges, g1)
    for rec in ket.log:
        assert rec["keep"] <= min(rec["m"], rec["n"])
        assert rec["keep"] <= rec["n"]


def test_structural_endpoints_by_hand_and_as_bounds():
    """The structural recursion that fixes which endpoint each compression SVDs (the endpoint with
    fewer rows 2 prod(other legs), ties to q[0]; bond <- min(dim chi_o, those rows, chi)), worked
    by hand on the chain 0-1-2 with fSim on (0,1), (1,2), (0,1), (1,2):
    (0,1): rows 2 vs 2, tie -> 0, bond min(4, 2) = 2;  (1,2): rows 4 vs 2 -> 2, bond min(4, 2) = 2;
    (0,1): rows 2 vs 4 -> 0, bond min(8, 2) = 2;       (1,2): rows 4 vs 2 -> 2, bond min(8, 2) = 2.
    A gate written (1,0) ties to its first qubit, 1. With chi = 1 every bond stays 1, so (1,2) sees
    rows 2 vs 2 and ties to 1: endpoints 0, 1, 0, 1. The recursion bounds every bond the evolution
    reaches, and the oracle compresses the endpoints it names."""
    from gen import Gate
    f = gen.fsim(np.pi / 2, np.pi / 6)
    chain = [(0, 1), (1, 2)]
    seq = [Gate(1, (0, 1), f), Gate(1, (1, 2), f), Gate(2, (0, 1), f), Gate(2, (1, 2), f)]
    assert tns.structural_svd_nodes(3, chain, seq, return_dims=True) == ([0, 2, 0, 2], [2, 2])
    assert tns.structural_svd_nodes(3, chain, [Gate(1, (1, 0), f)]) == [1]
    assert tns.structural_svd_nodes(3, chain, seq, chi=1, return_dims=True) == ([0, 1, 0, 1], [1, 1])
    g = gen.grid(3, 4)
    gates = gen.rqc(g, 6, gen.rng(41, 1), twoq="haar", oneq="haar")
    nodes, dims = tns.structural_svd_nodes(g.n, g.edges, gates, return_dims=True)
    ket = tns.evolve_ket(g.n, g.edges, gates)
    assert all(b <= d for b, d in zip(ket.bonds(), dims))
    assert [rec["svd_node"] for rec in ket.log] == nodes


def test_capped_fsim_compressions_meet_degenerate_spectra():
    """fSim(pi/2, phi) has a flat operator-Schmidt spectrum, so after a compression the SVD'd
    endpoint stays an isometry: later compressions of it see equal singular values, and a chi cap
    below them keeps an arbitrary half of a degenerate subspace. Truncated amplitudes of such
    circuits are therefore not unique (any SVD routine may pick another half); exact comparisons
    need untruncated runs or cuts inside a gap."""
    w = gen.regular3_family(count=32, n_bits=1)[7]
    g1, _ = tns.split_gates(w.gates, w.split)
    ket = tns.evolve_ket(w.graph.n, w.graph.edges, g1, chi=2)
    degenerate = [rec for rec in ket.log
                  if rec["keep"] < len(rec["s"]) and rec["s"][rec["keep"]] > 1e-12 * rec["s"][0]
                  and rec["s"][rec["keep"] - 1] / rec["s"][rec["keep"]] < 1 + 1e-9]
    assert len(degenerate) > 0
    _, _, chi_o = tns.gate_split(gen.fsim(np.pi / 2, np.pi / 6))
    s = np.linalg.svd(gen.fsim(np.pi / 2, np.pi / 6).reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4),
                      compute_uv=False)
    assert chi_o == 4 and np.allclose(s, s[0])


def test_graph_state_closed_form_at_scale():
    """H on every qubit, then CZ on every edge: a(s) = 2^{-n/2} (-1)^{sum_edges s_i s_j}, at 53 and 104 qubits."""
    for g in (gen.staggered(6, 9, remove_seed=gen.BASE_SEED + 3), gen.staggered(8, 13)):
        gates = gen.graph_state_circuit(g)
        bits = gen.bitstrings(g.n, 3, gen.rng(5, 2))
        for split in (0, 1):
            a, _ = tns.amplitudes(g.n, g.edges, gates, bits, split)
            par = np.array([sum(int(b[u]) * int(b[v]) for u, v in g.edges) for b in bits])
            expect = 2.0 ** (-g.n / 2) * (-1.0) ** par
            assert np.max(np.abs(a - expect)) / 2.0 ** (-g.n / 2) < 1e-10


def test_mirror_circuit_is_delta():
    w = gen.workload("grid12", n_bits=1)
    gates = gen.mirror_circuit(w.gates)
    bits = np.vstack([np.zeros(12, np.uint8), gen.bitstrings(12, 5, gen.rng(3, 2))])
    a, _ = tns.amplitudes(12, w.graph.edges, gates, bits, w.depth)
    assert abs(a[0] - 1) < 1e-12 and np.max(np.abs(a[1:])) < 1e-12
    g53 = gen.staggered(6, 9, remove_seed=gen.BASE_SEED + 3)
    gates = gen.mirror_circuit(gen.rqc(g53, 1, gen.rng(9, 1)))
    bits = np.vstack([np.zeros(53, np.uint8), gen.bitstrings(53, 2, gen.rng(9, 2))])
    a, _ = tns.amplitudes(53, g53.edges, gates, bits, 1)
    assert abs(a[0] - 1) < 1e-12 and np.max(np.abs(a[1:])) < 1e-12


def test_truncation_changes_only_with_chi():
    """chi at or above the untruncated bonds changes nothing; a small chi does."""
    w = gen.workload("grid12", n_bits=8)
    psi = sv.run(12, w.gates)
    ref = sv.amplitudes(psi, w.bits)
    a, _ = tns.amplitudes(12, w.graph.edges, w.gates, w.bits, w.split, chi=64)
    assert rel_err(a, ref) < 1e-12
    a2, _ = tns.amplitudes(12, w.graph.edges, w.gates, w.bits, w.split, chi=2)
    assert rel_err(a2, ref) > 1e-3


# ---------------------------------------------------------------- path scores
def test_path_subset_dp_equals_bruteforce():
    rng = np.random.default_rng(3)
    for n in (4, 5, 6, 7):
        edges = set()
        for i in range(1, n):
            edges.add((int(rng.integers(i)), i))
        for _ in range(n):
            u, v = sorted(rng.choice(n, 2, replace=False))
            edges.add((int(u), int(v)))
        edges = sorted(edges)
        dims = rng.integers(2, 9, size=len(edges))
        assert opath.bruteforce_optimum(n, edges, dims) == opath.subset_dp_optimum(n, edges, dims)


def test_path_cost_by_hand():
    # path graph 0-1-2 with dims 3 (edge 0-1) and 5 (edge 1-2)
    edges, dims = [(0, 1), (1, 2)], [3, 5]
    assert opath.score([0, 1, 2], edges, dims) == 3 * 5 + 5
    assert opath.score([1, 0, 2], edges, dims) == 3 * 5 + 5
    assert opath.score([0, 2, 1], edges, dims) == 3 * 5 + 3 * 5
