"""The gate programs checked on the CPU: the program tn_evolve_two_sided builds for each half
(tn_program_inspect, host only) is run by a NumPy model of the gate kernel's entry definition
stated in include/tn.h (the gate's P and Q on the physical index, the SVD of the named endpoint,
the keep rule, zero padding to the structural bond, absorption of S V^H into the other endpoint),
starting from the oracle's product states. The amplitudes of the resulting ket and bra must be
those of the oracle run with the same compression: the one-sided form of Eqs. svd/svd2, and the
two-sided form (singular values of the local product A^k A^l^T), which the library runs as two
entries per gate. The model restates the entry definition; it shares no code with the library."""
import numpy as np
import pytest

import gen
from oracle import statevector as sv
from oracle import tns as otns


@pytest.fixture(scope="module")
def tn(repo_root):
    from paper_2011_02621_gb300 import build
    build.build()
    from paper_2011_02621_gb300 import tn as _tn
    return _tn


def _entry(t, d):
    """One two-qubit entry on the TNS t (node tensors [sigma, legs in increasing edge id])."""
    k, l, e = d["k"], d["l"], d["edge"]
    pk, pl = 1 + d["pk"], 1 + d["pl"]
    assert t.legs[k][d["pk"]] == e and t.legs[l][d["pl"]] == e
    assert t.A[k].shape[pk] == d["din"] and t.A[l].shape[pl] == d["din"]
    chi_o, n, dout = d["chi_o"], d["n"], d["dout"]
    assert n == d["din"] * chi_o
    # X = P A: sum over the input value s of the physical index; the shared leg becomes
    # (a_old, a) at index a_old * chi_o + a (Eqs. result1/result2)
    X = []
    for A, P, pos in ((t.A[k], d["P"], pk), (t.A[l], d["Q"], pl)):
        Y = np.tensordot(P[:, :, :chi_o], A, axes=(1, 0))           # [s', a, legs...]
        Y = np.moveaxis(Y, 1, pos + 1)                              # a right after the shared leg
        shape = list(A.shape)
        shape[pos] *= chi_o
        X.append(Y.reshape(shape))
    Xk, Xl = X
    assert Xk[0].size * 2 == d["m_k"] * n and Xl[0].size * 2 == d["m_l"] * n
    if d["sv_is_k"]:
        Xs, ps, Xo, po = Xk, pk, Xl, pl
    else:
        Xs, ps, Xo, po = Xl, pl, Xk, pk
    Ms = np.moveaxis(Xs, ps, -1)
    rest = Ms.shape[:-1]
    U, S, Vh = np.linalg.svd(Ms.reshape(-1, n), full_matrices=False)
    keep = int(np.sum(S > d["cutoff"] * S[0])) if S.size and S[0] > 0 else 0
    keep = min(keep, dout)
    Un = np.zeros((U.shape[0], dout), complex)
    Un[:, :keep] = U[:, :keep]
    Vp = np.zeros((dout, n), complex)
    Vp[:keep] = S[:keep, None] * Vh[:keep]
    As = np.moveaxis(Un.reshape(rest + (dout,)), -1, ps)
    Ao = np.moveaxis(np.tensordot(Xo, Vp, axes=(po, 1)), -1, po)
    if d["sv_is_k"]:
        t.A[k], t.A[l] = As, Ao
    else:
        t.A[k], t.A[l] = Ao, As


def _run(prog, n, edges, bits=None):
    t = otns.TNS(n, edges, bits)
    for d in prog:
        if d["op"] == 1:
            t.A[d["k"]] = np.tensordot(d["u"], t.A[d["k"]], axes=(1, 0))
        else:
            _entry(t, d)
    return t


def _amplitudes(tn, w, split, chi, cutoff, compress):
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_set_compression(c, compress)
    ket_prog = tn.tn_program_inspect(c, split, chi, cutoff, 0)
    bra_prog = tn.tn_program_inspect(c, split, chi, cutoff, 1)
    ket = _run(ket_prog, w.graph.n, w.graph.edges)
    out = np.array([otns.overlap_amplitude(ket, _run(bra_prog, w.graph.n, w.graph.edges, b)) for b in w.bits])
    return out, ket_prog, bra_prog


def _rel(a, ref):
    return float(np.max(np.abs(a - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2)))


def _haar_grid_case(seed, n_bits=4):
    """A 3x4 grid with Haar-random two-qubit gates (generic singular value spectra, so a capped
    bond is cut inside a gap rather than through a degenerate multiplet, and two correct
    implementations keep the same subspace)."""
    import types
    g = gen.grid(3, 4)
    gates = gen.rqc(g, 8, gen.rng(seed, 1), twoq="haar", oneq="haar")
    return types.SimpleNamespace(graph=g, gates=gates, bits=gen.bitstrings(12, n_bits, gen.rng(seed, 2)))


@pytest.mark.parametrize("compress", ["one_sided", "two_sided"])
@pytest.mark.parametrize("split", [0, 3, 5, 8])
def test_untruncated_programs_give_the_statevector(tn, compress, split):
    w = gen.workload("grid12", n_bits=6)
    ref = sv.amplitudes(sv.run(12, w.gates), w.bits)
    a, _, _ = _amplitudes(tn, w, split, 0, 1e-12, compress)
    assert _rel(a, ref) < 1e-12


def test_untruncated_two_sided_program_on_a_random_regular_graph(tn):
    w = gen.regular3_family(count=1, depth=6, n_bits=4)[0]
    n = w.graph.n
    assert n <= 24
    ref = sv.amplitudes(sv.run(n, w.gates), w.bits)
    a, _, _ = _amplitudes(tn, w, w.split, 0, 1e-12, "two_sided")
    assert _rel(a, ref) < 1e-11


@pytest.mark.parametrize("compress", ["one_sided", "two_sided"])
@pytest.mark.parametrize("split,chi", [(0, 4), (8, 4), (8, 8), (4, 2)])
@pytest.mark.parametrize("seed", [43, 44])
def test_truncated_programs_match_the_oracle(tn, compress, split, chi, seed):
    w = _haar_grid_case(seed)
    ref, _ = otns.amplitudes(12, w.graph.edges, w.gates, w.bits, split, chi, 1e-12, compress=compress)
    a, _, _ = _amplitudes(tn, w, split, chi, 1e-12, compress)
    assert _rel(a, ref) < 1e-10


def test_two_sided_and_one_sided_differ_when_truncated(tn):
    """The comparison above can tell the forms apart: with truncation they give different
    amplitudes, and the state vector is closer to the two-sided ones on this circuit."""
    w = _haar_grid_case(43)
    exact = sv.amplitudes(sv.run(12, w.gates), w.bits)
    one, _, _ = _amplitudes(tn, w, 8, 8, 1e-12, "one_sided")
    two, _, _ = _amplitudes(tn, w, 8, 8, 1e-12, "two_sided")
    assert _rel(one, two) > 0.1
    assert _rel(two, exact) < _rel(one, exact)


def test_two_sided_program_structure(tn):
    """Two entries per two-qubit gate: the gate with the other endpoint decomposed whole (cutoff
    0, bond min(n, its rows), no chi cap), then a one-term identity decomposing the endpoint with
    fewer rows under the keep rule and the chi cap. The structural bonds after each half equal
    the one-sided program's, so plans have the same shapes."""
    w = gen.workload("syc53", n_bits=1)
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    one = [tn.tn_program_inspect(c, w.split, w.chi, w.cutoff, s) for s in (0, 1)]
    lay1 = tn.tn_plan_inspect(c, w.split, w.chi, w.cutoff)[0]
    tn.tn_set_compression(c, "two_sided")
    two = [tn.tn_program_inspect(c, w.split, w.chi, w.cutoff, s) for s in (0, 1)]
    lay2 = tn.tn_plan_inspect(c, w.split, w.chi, w.cutoff)[0]
    eye = np.zeros((2, 2, 4), complex)
    eye[0, 0, 0] = eye[1, 1, 0] = 1
    for p1, p2 in zip(one, two):
        g1 = [d for d in p1 if d["op"] == 2]
        g2 = [d for d in p2 if d["op"] == 2]
        assert len(g2) == 2 * len(g1)
        for d, a, b in zip(g1, g2[0::2], g2[1::2]):
            assert (a["k"], a["l"], a["edge"]) == (b["k"], b["l"], b["edge"]) == (d["k"], d["l"], d["edge"])
            assert np.array_equal(a["P"], d["P"]) and np.array_equal(a["Q"], d["Q"]) and a["chi_o"] == d["chi_o"]
            assert a["sv_is_k"] == 1 - d["sv_is_k"] and b["sv_is_k"] == d["sv_is_k"]
            assert a["cutoff"] == 0.0 and b["cutoff"] == d["cutoff"]
            rows_other = a["m_k"] if a["sv_is_k"] else a["m_l"]
            assert a["dout"] == min(a["n"], rows_other)
            assert b["chi_o"] == 1 and b["din"] == a["dout"] and np.array_equal(b["P"], eye)
            assert np.array_equal(b["Q"], eye)
            assert b["dout"] == d["dout"]
        t1 = [d for d in p1 if d["op"] == 1]
        t2 = [d for d in p2 if d["op"] == 1]
        assert [d["k"] for d in t1] == [d["k"] for d in t2]
        assert all(np.array_equal(x["u"], y["u"]) for x, y in zip(t1, t2))
    assert np.array_equal(lay1["ket_dims"], lay2["ket_dims"]) and np.array_equal(lay1["bra_dims"], lay2["bra_dims"])


def test_a_program_truncating_its_first_entry_is_caught(tn):
    """A mistaken two-sided program that caps the whole decomposition at chi as well no longer
    matches the oracle: the comparison above would catch it."""
    w = _haar_grid_case(44)
    ref, _ = otns.amplitudes(12, w.graph.edges, w.gates, w.bits, 8, 4, 1e-12, compress="two_sided")
    c = tn.tn_build(12, w.graph.edges, w.gates)
    tn.tn_set_compression(c, "two_sided")
    ket_prog = tn.tn_program_inspect(c, 8, 4, 1e-12, 0)
    bad = []
    for i, d in enumerate(ket_prog):
        d = dict(d)
        if d["op"] == 2 and d["cutoff"] == 0.0:      # a first entry
            d["dout"] = min(d["dout"], 2)
            nxt = ket_prog[i + 1]
            assert nxt["din"] >= d["dout"]
        bad.append(d)
    # the entries after a capped one see narrower bonds: rebuild their din / n from the state
    t = otns.TNS(12, w.graph.edges)
    for d in bad:
        if d["op"] == 1:
            t.A[d["k"]] = np.tensordot(d["u"], t.A[d["k"]], axes=(1, 0))
            continue
        din = t.A[d["k"]].shape[1 + d["pk"]]
        d = dict(d, din=din, n=din * d["chi_o"], m_k=t.A[d["k"]].size // din, m_l=t.A[d["l"]].size // din)
        d["dout"] = min(d["dout"], d["n"], d["m_k"] if d["sv_is_k"] else d["m_l"])
        _entry(t, d)
    bra = _run(tn.tn_program_inspect(c, 8, 4, 1e-12, 1), 12, w.graph.edges, w.bits[0])
    assert abs(otns.overlap_amplitude(t, bra) - ref[0]) > 1e-3 * np.sqrt(np.mean(np.abs(ref) ** 2))


def test_unknown_compression_mode_is_refused(tn):
    w = gen.workload("grid12", n_bits=1)
    c = tn.tn_build(12, w.graph.edges, w.gates)
    with pytest.raises(ValueError):
        tn.tn_set_compression(c, "three_sided")
    assert tn.LIB.tn_set_compression(c.ptr, 2) == tn.TN_ERR_ARG


@pytest.mark.parametrize("compress", ["one_sided", "two_sided"])
@pytest.mark.parametrize("layers", [1, 2])
@pytest.mark.parametrize("chi,split", [(0, 4), (4, 8), (4, 0)])
def test_programs_feed_the_compiled_plan(tn, compress, layers, chi, split):
    """The two host-side models chained: the node tensors the gate programs leave (at exactly the
    plan's structural bonds, in the halves' slots) contracted by the compiled plan's steps give
    the oracle's amplitude for the same compression (the state vector's when nothing is cut)."""
    from tests.test_plan_emulation import _execute, _place
    w = _haar_grid_case(44, n_bits=3)
    c = tn.tn_build(12, w.graph.edges, w.gates)
    tn.tn_set_compression(c, compress)
    layout, steps, tab = tn.tn_plan_inspect(c, split, chi, 1e-12, layers=layers, merge=False)
    ket = _run(tn.tn_program_inspect(c, split, chi, 1e-12, 0), 12, w.graph.edges)
    assert ket.bonds() == list(layout["ket_dims"])
    kbuf = _place(ket, layout["ket_dims"], layout["ket_off"], layout["ket_half_elems"])
    ref, _ = otns.amplitudes(12, w.graph.edges, w.gates, w.bits, split, chi, 1e-12, compress=compress)
    if chi == 0:
        assert _rel(ref, sv.amplitudes(sv.run(12, w.gates), w.bits)) < 1e-12
    bra_prog = tn.tn_program_inspect(c, split, chi, 1e-12, 1)
    got = []
    for b in w.bits:
        bra = _run(bra_prog, 12, w.graph.edges, b)
        assert bra.bonds() == list(layout["bra_dims"])
        got.append(_execute(layout, steps, tab, kbuf, _place(bra, layout["bra_dims"], layout["bra_off"],
                                                             layout["bra_half_elems"])))
    assert _rel(np.array(got), ref) < 1e-10


def test_program_inspection_arguments(tn):
    w = gen.workload("grid12", n_bits=1)
    c = tn.tn_build(12, w.graph.edges, w.gates)
    n = tn.C.c_int64()
    assert tn.LIB.tn_program_inspect(c.ptr, 4, 0, 1e-12, 2, None, None, tn.C.byref(n)) == tn.TN_ERR_ARG
    assert tn.LIB.tn_program_inspect(c.ptr, -1, 0, 1e-12, 0, None, None, tn.C.byref(n)) == tn.TN_ERR_ARG
    assert tn.LIB.tn_program_inspect(None, 4, 0, 1e-12, 0, None, None, tn.C.byref(n)) == tn.TN_ERR_ARG
    # every gate in the ket: the bra program is empty, the ket holds all 34 two-qubit gates
    assert tn.tn_program_inspect(c, w.depth, 0, 1e-12, 1) == []
    assert sum(d["op"] == 2 for d in tn.tn_program_inspect(c, w.depth, 0, 1e-12, 0)) == 34
