"""Planted mistakes in the oracle (on the CPU) must fail its pins.

Each test patches one plausible error into the oracle and checks that the
state-vector pin or a closed form then rejects it, so that a pin set that
cannot see a dropped transpose, a stray conjugate or a mis-merged bond index
would itself be caught."""
import math

import numpy as np
import pytest

import gen
from oracle import path as opath
from oracle import statevector as sv
from oracle import tns


def _err_vs_statevector(twoq="fsim"):
    w = gen.workload("grid12", n_bits=8)
    if twoq != "fsim":
        w.gates = gen.rqc(w.graph, w.depth, gen.rng(77, 1), twoq=twoq)
    psi = sv.run(12, w.gates)
    ref = sv.amplitudes(psi, w.bits)
    # split after cycle 6: the C and D edges get two gates in the ket half
    a, _ = tns.amplitudes(12, w.graph.edges, w.gates, w.bits, 6)
    return float(np.max(np.abs(a - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2)))


def test_unpatched_oracle_passes():
    assert _err_vs_statevector() < 1e-12
    assert _err_vs_statevector("haar") < 1e-12


def test_bra_without_transpose_is_caught(monkeypatch):
    orig = tns.TNS.apply

    def no_transpose(self, gate, chi=0, cutoff=1e-12, transpose=False, svd_node=None, compress="one_sided"):
        return orig(self, gate, chi, cutoff, transpose=False, svd_node=svd_node, compress=compress)
    monkeypatch.setattr(tns.TNS, "apply", no_transpose)
    assert _err_vs_statevector() > 1e-3


def test_conjugated_overlap_is_caught(monkeypatch):
    orig = tns.overlap_node
    monkeypatch.setattr(tns, "overlap_node", lambda A, B: orig(A, B.conj()))
    assert _err_vs_statevector() > 1e-3


def test_bond_index_order_mismatch_is_caught(monkeypatch):
    orig = tns.TNS._apply_half
    calls = {"n": 0}

    def swapped(T, P, pos):
        calls["n"] += 1
        if calls["n"] % 2 == 0:           # second endpoint merges (s, a) instead of (a, s)
            out = np.tensordot(P, T, axes=(1, 0))
            out = np.moveaxis(out, 1, pos)
            shape = list(T.shape)
            shape[pos] *= P.shape[2]
            return out.reshape(shape)
        return orig(T, P, pos)
    monkeypatch.setattr(tns.TNS, "_apply_half", staticmethod(swapped))
    assert _err_vs_statevector() > 1e-3


def test_gate_split_without_regrouping_is_caught(monkeypatch):
    def bad_split(m, rel=1e-12):
        R = np.asarray(m).reshape(4, 4)           # forgot the (k',k) x (l',l) regrouping
        U, S, Vh = np.linalg.svd(R)
        c = int(np.sum(S > rel * S[0]))
        sq = np.sqrt(S[:c])
        return (U[:, :c] * sq).reshape(2, 2, c), (sq[:, None] * Vh[:c]).T.reshape(2, 2, c), c
    monkeypatch.setattr(tns, "gate_split", bad_split)
    assert _err_vs_statevector("haar") > 1e-3


def test_cost_counting_shared_legs_twice_is_caught(monkeypatch):
    def bad_cost(mask, i, edges, dims):
        c = 1
        for e in opath.open_legs(mask, edges):
            c *= int(dims[e])
        for e, (u, v) in enumerate(edges):
            if i in (u, v):
                c *= int(dims[e])
        return c
    monkeypatch.setattr(opath, "cost", bad_cost)
    edges, dims = [(0, 1), (1, 2)], [3, 5]
    assert opath.score([0, 1, 2], edges, dims) != 3 * 5 + 5
