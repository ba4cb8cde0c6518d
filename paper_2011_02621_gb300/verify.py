"""Verification of random-circuit runs from computed amplitudes.

* Eq. fidelity: the fidelity of a noisy device running the circuit, estimated as the product of
  (1 - error rate) over its gates and over its qubits' readouts; the defaults are the single-qubit,
  two-qubit and readout error rates the paper quotes for the Sycamore processor (0.16%, 0.62%,
  3.8%).
* The smallest number of bitstrings N_s that keeps that fidelity three statistical standard
  deviations (1/sqrt(N_s) each) above zero: N_s >= (3 / F)^2.
* Linear cross-entropy benchmarking over computed amplitudes: 2^n <|a(s)|^2> - 1 over the sampled
  bitstrings s; its expectation is the fidelity of the sampler (1 for samples of the ideal
  distribution of a deep random circuit, whose probabilities follow Porter-Thomas statistics; 0
  for uniformly random bitstrings).
These use only amplitudes the library has already computed; nothing here touches the device."""
from __future__ import annotations

import math
from typing import Iterable

import numpy as np


def circuit_fidelity(gates: Iterable, n_qubits: int, e1: float = 0.0016, e2: float = 0.0062,
                     eq: float = 0.038) -> float:
    """Eq. fidelity for ``gates`` (objects with a ``qubits`` tuple of length 1 or 2) on
    ``n_qubits`` read-out qubits."""
    n1 = n2 = 0
    for g in gates:
        if len(g.qubits) == 1:
            n1 += 1
        elif len(g.qubits) == 2:
            n2 += 1
        else:
            raise ValueError("gates act on one or two qubits")
    return (1.0 - e1) ** n1 * (1.0 - e2) ** n2 * (1.0 - eq) ** n_qubits


def required_bitstrings(fidelity: float, sigmas: float = 3.0) -> int:
    """Smallest N_s with fidelity >= sigmas / sqrt(N_s)."""
    if not fidelity > 0:
        raise ValueError("fidelity must be positive")
    return int(math.ceil((sigmas / fidelity) ** 2 - 1e-9))


def linear_xeb(amplitudes, n_qubits: int) -> float:
    """2^n <|a|^2> - 1 over the given amplitudes (one per sampled bitstring)."""
    a = np.asarray(amplitudes)
    if a.size == 0:
        raise ValueError("no amplitudes")
    return float(2.0 ** n_qubits * np.mean(np.abs(a) ** 2) - 1.0)
