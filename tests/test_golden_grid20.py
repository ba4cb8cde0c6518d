"""The stored oracle amplitudes of the 4x5 grid at 14 cycles (tests/golden/grid20_oracle.json,
written by tests/golden/make_grid20_oracle.py from the oracle's double-layer contraction) pinned
to something other than the oracle: the brute-force 2^20 state vector, and the bitstrings to the
seeded generator."""
import json
import os

import numpy as np

import gen
from oracle import statevector as sv

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "grid20_oracle.json")


def test_grid20_golden_amplitudes_equal_the_statevector():
    d = json.load(open(GOLDEN))
    bits = np.array(d["bits"], dtype=np.uint8)
    w = gen.workload("grid20", n_bits=len(bits))
    assert np.array_equal(bits, w.bits)
    amps = np.array([complex(r, i) for r, i in d["amplitudes"]])
    ref = sv.amplitudes(sv.run(20, w.gates), bits)
    assert np.max(np.abs(amps - ref)) <= 1e-12 * np.sqrt(np.mean(np.abs(ref) ** 2))
