"""The verification layer (Eq. fidelity, the required number of bitstrings, linear XEB) against
hand-worked values and the statistics of exact amplitudes (CPU, oracle state vectors)."""
import math

import numpy as np
import pytest

import gen
from oracle import statevector as sv
from paper_2011_02621_gb300 import verify


def test_fidelity_by_hand():
    """Two single-qubit gates, one two-qubit gate, three qubits read out:
    (1 - 0.0016)^2 (1 - 0.0062) (1 - 0.038)^3 = 0.99680256 * 0.9938 * 0.890277128."""
    gates = [gen.Gate(1, (0,), np.eye(2)), gen.Gate(1, (1,), np.eye(2)), gen.Gate(1, (0, 1), np.eye(4))]
    f = verify.circuit_fidelity(gates, 3)
    assert abs(f - 0.99680256 * 0.9938 * 0.890277128) < 1e-12
    assert verify.circuit_fidelity([], 0) == 1.0
    with pytest.raises(ValueError):
        verify.circuit_fidelity([gen.Gate(1, (0, 1, 2), np.eye(8))], 3)


def test_required_bitstrings():
    """N_s >= (3 / F)^2: F = 0.3 needs 100 bitstrings; F = 0.01 needs 90000."""
    assert verify.required_bitstrings(0.3) == 100
    assert verify.required_bitstrings(0.01) == 90000
    assert verify.required_bitstrings(1.0) == 9
    with pytest.raises(ValueError):
        verify.required_bitstrings(0.0)


def test_fidelity_falls_with_depth_on_the_53_qubit_grid():
    g = gen.staggered(6, 9, remove_seed=gen.BASE_SEED + 3)
    fs = [verify.circuit_fidelity(gen.rqc(g, d, gen.rng(1, 1)), g.n) for d in (2, 6, 10, 14)]
    assert all(a > b for a, b in zip(fs, fs[1:]))
    ns = [verify.required_bitstrings(f) for f in fs]
    assert all(a < b for a, b in zip(ns, ns[1:]))


def test_linear_xeb_ideal_samples_and_uniform_bitstrings():
    """Deep 12-qubit random circuit: bitstrings drawn from its own output distribution give
    2^n <p> - 1 = 2^n sum p^2 - 1, about 1 (Porter-Thomas); uniformly random ones give about 0;
    both against the exact sums over all 2^n bitstrings."""
    w = gen.workload("grid12", n_bits=1)
    psi = sv.run(12, w.gates)
    allbits = gen.all_bitstrings(12)
    amps = sv.amplitudes(psi, allbits)
    p = np.abs(amps) ** 2                                    # in the order of allbits
    exact_ideal = 2 ** 12 * float(np.sum(p ** 2)) - 1
    assert abs(exact_ideal - 1) < 0.3
    assert abs(verify.linear_xeb(amps, 12)) < 1e-12          # uniform over all: exactly 0
    rng = np.random.default_rng(3)
    idx = rng.choice(len(p), size=20000, p=p / p.sum())
    est = verify.linear_xeb(amps[idx], 12)
    assert abs(est - exact_ideal) < 5 * math.sqrt(2 ** 24 * np.sum(p ** 3) / 20000)
    with pytest.raises(ValueError):
        verify.linear_xeb([], 12)
