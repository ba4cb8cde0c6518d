"""Writes grid20_oracle.json: the oracle's amplitudes of the first 16 bitstrings of the 4x5 grid,
14-cycle workload (untruncated), from the double-layer contraction of its two-sided evolution
(every ket and bra tensor a node of its own, the oracle's own pairwise order). Calls only oracle/
and gen/. Run from the repository root: python tests/golden/make_grid20_oracle.py"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gen  # noqa: E402
from oracle import tns  # noqa: E402


def main(n_bits=16):
    w = gen.workload("grid20", n_bits=n_bits)
    g1, g2 = tns.split_gates(w.gates, w.split)
    ket = tns.evolve_ket(w.graph.n, w.graph.edges, g1, w.chi, w.cutoff)
    amps = []
    for b in w.bits:
        bra = tns.evolve_bra(w.graph.n, w.graph.edges, g2, b, w.chi, w.cutoff)
        a = tns.double_layer_amplitude(ket, bra)
        amps.append([a.real, a.imag])
    out = {"workload": "grid20 (4x5 grid, 14 cycles, split 7, untruncated), first 16 bitstrings of gen.workload",
           "method": "oracle.tns.double_layer_amplitude of the two-sided evolution",
           "bits": [[int(x) for x in b] for b in w.bits], "amplitudes": amps}
    with open(os.path.join(HERE, "grid20_oracle.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
