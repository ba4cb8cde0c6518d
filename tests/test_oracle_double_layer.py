"""The double-layer contraction of the oracle (ket and bra tensors as separate nodes joined by
their physical index; the sums of Eq. overlap grouped differently) against the state vector and
the overlap-network contraction, with a planted mistake that must fail."""
import numpy as np
import pytest

import gen
from oracle import statevector as sv
from oracle import tns


def _amps(w, split, fn, chi=0):
    g1, g2 = tns.split_gates(w.gates, split)
    ket = tns.evolve_ket(w.graph.n, w.graph.edges, g1, chi)
    out = []
    for b in w.bits:
        bra = tns.evolve_bra(w.graph.n, w.graph.edges, g2, b, chi)
        out.append(fn(ket, bra))
    return np.array(out)


@pytest.mark.parametrize("split", [0, 4, 8])
def test_double_layer_equals_statevector(split):
    w = gen.workload("grid12", n_bits=4)
    ref = sv.amplitudes(sv.run(12, w.gates), w.bits)
    a = _amps(w, split, tns.double_layer_amplitude)
    assert np.max(np.abs(a - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2)) < 1e-12


def test_double_layer_equals_statevector_on_a_random_graph():
    g = gen.random_regular3(12, gen.rng(8, 0))
    gates = gen.rqc(g, 6, gen.rng(8, 1), twoq="haar", oneq="haar")
    bits = gen.bitstrings(12, 3, gen.rng(8, 2))
    w = gen.Workload.__new__(gen.Workload)
    w.graph, w.gates, w.bits = g, gates, bits
    ref = sv.amplitudes(sv.run(12, gates), bits)
    a = _amps(w, 3, tns.double_layer_amplitude)
    assert np.max(np.abs(a - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2)) < 1e-12


def test_double_layer_equals_overlap_network_when_truncated():
    """With chi = 2 the amplitudes differ from the state vector, but both groupings of the sums
    contract the same truncated tensors."""
    w = gen.workload("grid12", n_bits=4)
    ref = sv.amplitudes(sv.run(12, w.gates), w.bits)
    a = _amps(w, 6, tns.double_layer_amplitude, chi=2)
    b = _amps(w, 6, tns.overlap_amplitude, chi=2)
    scale = np.sqrt(np.mean(np.abs(b) ** 2))
    assert np.max(np.abs(a - b)) / scale < 1e-12
    assert np.max(np.abs(b - ref)) / scale > 1e-3        # the truncation is real


def test_conjugated_bra_layer_is_caught(monkeypatch):
    w = gen.workload("grid12", n_bits=3)
    ref = sv.amplitudes(sv.run(12, w.gates), w.bits)
    orig = tns.double_layer_amplitude

    def planted(ket, bra):
        bra.A = [x.conj() for x in bra.A]
        return orig(ket, bra)
    a = _amps(w, 4, planted)
    assert np.max(np.abs(a - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2)) > 1e-3
