"""Writes reg3_n24_statevector.json: exact amplitudes <s|U|0...0> of the first 24-qubit circuit of
the random 3-regular family (12 cycles: Haar SU(2) on every qubit, then fSim(pi/2, pi/6) on one
edge colour class), for its first 8 seeded bitstrings, from the 2^24 state vector (the definition
of the amplitude; the untruncated method reaches it exactly). Calls only the oracle and the seeded
generators. Run from the repository root: python tests/golden/make_reg3_statevector.py"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import gen                                   # noqa: E402
from oracle import statevector as sv         # noqa: E402


def main():
    w = gen.regular3_family(count=32, n_bits=8)[0]
    psi = sv.run(w.graph.n, w.gates)
    a = sv.amplitudes(psi, w.bits)
    out = {"workload": w.name, "n_qubits": w.graph.n, "depth": w.depth, "n_bits": 8,
           "source": "2^24 state vector (oracle.statevector), complex128",
           "re": [float(x.real) for x in a], "im": [float(x.imag) for x in a]}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "reg3_n24_statevector.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
