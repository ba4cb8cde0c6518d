"""The plan compiler checked on the CPU: the compiled steps of a plan (tn_plan_inspect, host
only) are executed by a NumPy model of the step definition stated in include/tn.h, on the
oracle's ket and bra tensors zero-padded to the plan's structural bonds, and must give the
oracle's amplitude. Covers the overlap network and the double-layer network (ket-only and
bra-only steps with the unit operand), every split of the 3x4 grid, cut plans (slice tables)
and the 53-qubit benchmark circuit. The model restates the step definition; it shares no code
with the library."""
import numpy as np
import pytest

import gen
from oracle import tns as otns


@pytest.fixture(scope="module")
def tn(repo_root):
    from paper_2011_02621_gb300 import build
    build.build()
    from paper_2011_02621_gb300 import tn as _tn
    return _tn


def _place(t, dims, offs, size):
    """Node tensors [sigma, legs in increasing edge id] at their item offsets, zero-padded."""
    buf = np.zeros(size, complex)
    for q in range(t.n):
        A = t.A[q]
        P = np.zeros((2,) + tuple(int(dims[e]) for e in t.legs[q]), complex)
        assert all(a <= b for a, b in zip(A.shape, P.shape))
        P[tuple(slice(0, s) for s in A.shape)] = A
        buf[offs[q]: offs[q] + P.size] = P.ravel()
    return buf


def _execute(layout, steps, tab, ket, bra):
    """One bitstring, all slices: the steps as the header defines them."""
    tab = tab.astype(np.int64)
    S, maxT = layout["n_slices"], layout["max_t"]
    unit = np.array([1, 0], complex)
    T = np.zeros((S, maxT), complex)
    for j, st in enumerate(steps):
        x_buf = unit if st["layer"] == 2 else ket
        y_buf = unit if st["layer"] == 1 else bra
        M, K, N = st["M"], st["K"], st["N"]
        ocol = tab[st["t_ocol"]: st["t_ocol"] + N]
        bka = tab[st["t_bka"]: st["t_bka"] + K] if j else np.zeros(1, np.int64)
        bkb = tab[st["t_bkb"]: st["t_bkb"] + K] if j else np.zeros(1, np.int64)
        bna = tab[st["t_bna"]: st["t_bna"] + N]
        bnb = tab[st["t_bnb"]: st["t_bnb"] + N]
        orow = np.zeros(M, np.int64)
        m = np.arange(M)
        for d, o in zip(reversed(st["rest_dim"]), reversed(st["rest_ostride"])):
            orow += (m % d) * o
            m //= d
        Tn = np.zeros_like(T)
        for item in range(S):
            x0 = st["ket_off"] + tab[st["t_sa"] + item]
            y0 = st["bra_off"] + tab[st["t_sb"] + item]
            Cm = np.zeros((len(bka), N), complex)
            for s in range(st["phys"]):
                Cm += x_buf[x0 + bka[:, None] + bna[None, :] + s * st["ket_sig"]] * \
                      y_buf[y0 + bkb[:, None] + bnb[None, :] + s * st["bra_sig"]]
            if j == 0:
                Tn[item, ocol] = Cm[0]
            else:
                out = T[item, : M * K].reshape(M, K) @ Cm
                Tn[item, (orow[:, None] + ocol[None, :]).ravel()] = out.ravel()
        T = Tn
    return T[:, 0].sum()


def _check(tn, name, split=None, n_bits=2, **opts):
    w = gen.workload(name, n_bits=n_bits)
    split = w.split if split is None else split
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates, allocator=None)
    layout, steps, tab = tn.tn_plan_inspect(c, split, 0, 1e-12, **opts)
    assert not layout["merged"] and len(steps) == layout["n_steps"]
    g1, g2 = otns.split_gates(w.gates, split)
    ket = otns.evolve_ket(w.graph.n, w.graph.edges, g1)
    kbuf = _place(ket, layout["ket_dims"], layout["ket_off"], layout["ket_half_elems"])
    for b in w.bits:
        bra = otns.evolve_bra(w.graph.n, w.graph.edges, g2, b)
        bbuf = _place(bra, layout["bra_dims"], layout["bra_off"], layout["bra_half_elems"])
        ref = otns.overlap_amplitude(ket, bra)
        assert abs(_execute(layout, steps, tab, kbuf, bbuf) - ref) < 1e-12 * abs(ref)
    return layout, steps


@pytest.mark.parametrize("split", [0, 3, 4, 8])
@pytest.mark.parametrize("layers", [1, 2])
def test_compiled_steps_give_the_oracle_amplitude(tn, split, layers):
    layout, steps = _check(tn, "grid12", split=split, layers=layers, merge=False)
    assert len(steps) == (2 if layers == 2 else 1) * 12
    assert all(s["layer"] == 0 for s in steps) if layers == 1 else {s["layer"] for s in steps} == {1, 2}


@pytest.mark.parametrize("layers,limit", [(1, 64), (2, 64), (2, 32)])
def test_compiled_slice_tables(tn, layers, limit):
    layout, _ = _check(tn, "grid12", split=4, n_bits=1, layers=layers, merge=False, max_intermediate=limit)
    assert layout["n_slices"] > 1 and layout["max_t"] <= limit


@pytest.mark.parametrize("layers", [1, 2])
def test_compiled_steps_of_the_53_qubit_circuit(tn, layers):
    layout, steps = _check(tn, "syc53", n_bits=1, layers=layers, merge=False)
    assert len(steps) == (106 if layers == 2 else 53)


def test_inspection_reports_merged_plans(tn):
    w = gen.workload("syc53", n_bits=1)
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates, allocator=None)
    layout, steps, _ = tn.tn_plan_inspect(c, w.split, w.chi, w.cutoff)
    assert layout["merged"] and len(steps) == 34 and layout["ket_elems"] > layout["ket_half_elems"]
