"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
the CPU oracle on the same seeded inputs."""
import numpy as np

import gen
from oracle import statevector as sv
from oracle import tns as otns

FP64_TOL = 1e-10     # |da| / rms|a| on the FP64 path
TC_TOL = 1e-5        # |da| / rms|a| on the complex64 and tensor-core paths


def rel_err(a, ref):
    a, ref = np.asarray(a), np.asarray(ref)
    return float(np.max(np.abs(a - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2)))


def gpu_amplitudes(tn, n, edges, gates, bits, split, chi=0, cutoff=1e-12, prec="fp64", **path_opts):
    c = tn.tn_build(n, edges, gates)
    tn.tn_evolve_two_sided(c, split, chi, cutoff)
    p = tn.tn_path(c, **path_opts)
    a = tn.tn_amplitudes(p, bits, prec)
    return a, c, p


def oracle_amplitudes(n, edges, gates, bits, split, chi=0, cutoff=1e-12, cuts=()):
    a, _ = otns.amplitudes(n, edges, gates, bits, split, chi, cutoff, cuts)
    return a


def statevector_amplitudes(n, gates, bits):
    return sv.amplitudes(sv.run(n, gates), bits)
