"""Brute-force state-vector simulation (oracle; test infrastructure only).

The amplitude the method computes is a(s) = <s| U_d ... U_1 |0...0> (the
problem statement of the paper: amplitudes of a random circuit started from
|0>^N and projected on the target bitstring s_1 ... s_N, two-sided evolution
paragraph and Fig. 2a). For small N this file computes it by storing all 2^N
complex128 coefficients and applying every gate in order.

Layout: the state is an N-dimensional array of shape (2,)*N whose axis q is
qubit q, so psi[s_0, ..., s_{N-1}] = <s|psi>. A two-qubit gate matrix m is
indexed [(s0' s1'), (s0 s1)] with q[0] the high bit.
"""
from __future__ import annotations

from typing import Iterable, Sequence

import numpy as np


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    return psi


def apply_gate(psi: np.ndarray, qubits: Sequence[int], m: np.ndarray) -> np.ndarray:
    k = len(qubits)
    op = np.asarray(m, dtype=np.complex128).reshape((2,) * (2 * k))
    out = np.tensordot(op, psi, axes=(list(range(k, 2 * k)), list(qubits)))
    return np.moveaxis(out, list(range(k)), list(qubits))


def run(n: int, gates: Iterable) -> np.ndarray:
    """Apply ``gates`` (objects with ``.qubits`` and ``.m``) in order to |0...0>."""
    psi = zero_state(n)
    for g in gates:
        psi = apply_gate(psi, g.qubits, g.m)
    return psi


def amplitudes(psi: np.ndarray, bits: np.ndarray) -> np.ndarray:
    """a(s) for each row s of the (B, N) 0/1 array ``bits``."""
    bits = np.asarray(bits, dtype=np.int64)
    return psi[tuple(bits.T)]


def unitary_bruteforce(n: int, gates: Iterable) -> np.ndarray:
    """Full 2^N x 2^N circuit matrix, built entry by entry (tiny N only).

    Basis index i has bit q equal to s_q. Used to pin ``run`` by an
    implementation that shares no tensor reshaping with it.
    """
    dim = 1 << n
    U = np.eye(dim, dtype=np.complex128)
    for g in gates:
        qs = list(g.qubits)
        k = len(qs)
        G = np.zeros((dim, dim), dtype=np.complex128)
        for col in range(dim):
            sub_in = 0
            for j, q in enumerate(qs):
                sub_in = (sub_in << 1) | ((col >> q) & 1)
            for sub_out in range(1 << k):
                row = col
                for j, q in enumerate(qs):
                    bit = (sub_out >> (k - 1 - j)) & 1
                    row = (row & ~(1 << q)) | (bit << q)
                G[row, col] += g.m[sub_out, sub_in]
        U = G @ U
    return U
