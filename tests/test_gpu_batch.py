"""Batched circuits of uneven shape in one graph launch, and the step-kernel autotuner.

The workload is the random 3-regular family: 32 circuits of 24..40 qubits, 12 cycles of Haar
SU(2) on every qubit then fSim(pi/2, pi/6) on one edge colour class, each circuit with the
largest bond cap chi in {2, 4, ...} whose path needs no cut at 2^24 elements per bitstring.
Capped there, the one-sided compressions of these circuits keep an arbitrary half of exactly
degenerate singular values (fSim(pi/2, .) has a flat operator-Schmidt spectrum; pinned on the
oracle), so their truncated amplitudes are not unique: the truncated batch is checked against
single tn_amplitudes calls (identical kernels, identical numbers) and across precisions (the
same FP64 truncation decisions). Parity with the oracle is checked where the result is unique:
untruncated, on the same family at 8 cycles, and on the 24-qubit, 12-cycle circuit against its
exact amplitudes from the 2^24 state vector (a stored fixture written by the oracle)."""
import json
import os

import numpy as np
import pytest

import gen
from tests.gpu_common import FP64_TOL, TC_TOL, oracle_amplitudes, rel_err

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2011_02621_gb300 import build
    build.build()
    from paper_2011_02621_gb300 import tn as _tn
    return _tn


@pytest.fixture(scope="module")
def family():
    return gen.regular3_family(count=32, n_bits=1024)


def _plans(tn, ws):
    out = []
    for w in ws:
        c, p, chi = tn.tn_build_largest_chi(w.graph.n, w.graph.edges, w.gates, w.split)
        out.append((w, c, p, chi))
    return out


def test_batch_matches_oracle_untruncated_family(tn):
    """24, 32 and 40 qubits at 8 cycles, untruncated, in one graph: FP64 equals the oracle, BF16x6
    is within 1e-5 of FP64, and every circuit's batch result equals its single call."""
    ws = [gen.regular3_family(count=32, depth=8, n_bits=48)[i] for i in (0, 16, 31)]
    plans = []
    for w in ws:
        c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
        tn.tn_evolve_two_sided(c, w.split)
        plans.append((w, c, tn.tn_path(c)))
    res = {}
    for prec in ("fp64", "bf16x6"):
        b = tn.tn_batch_create([p for _, _, p in plans], [w.bits for w in ws], prec)
        tn.tn_batch_run(b)
        res[prec] = b.split(tn.tn_batch_read(b))
        for (w, c, p), g in zip(plans, res[prec]):
            assert np.array_equal(g, tn.tn_amplitudes(p, w.bits, prec)), (w.name, prec)
        tn.tn_batch_free(b)
    for (w, c, p), g64, gtc in zip(plans, res["fp64"], res["bf16x6"]):
        ref = oracle_amplitudes(w.graph.n, w.graph.edges, w.gates, w.bits[:3], w.split)
        assert rel_err(g64[:3], ref) < FP64_TOL, w.name
        assert rel_err(gtc, g64) < TC_TOL, w.name


def test_untruncated_24_qubits_12_cycles_matches_state_vector(tn):
    """The 24-qubit circuit of the family, untruncated (intermediates up to 2^29, cut to 2^26):
    the slices, summed in FP64, give the exact amplitudes."""
    fx = json.load(open(os.path.join(HERE, "golden", "reg3_n24_statevector.json")))
    w = gen.regular3_family(count=32, n_bits=fx["n_bits"])[0]
    assert w.name == fx["workload"]
    ref = (np.asarray(fx["re"]) + 1j * np.asarray(fx["im"]))[:2]
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, 0, 1e-12)
    p = tn.tn_path(c, max_intermediate=1 << 26, mem_budget_bytes=16.0 * 2 ** 30)
    assert p.info["n_slices"] > 1
    b = tn.tn_batch_create([p], [w.bits[:2]], "fp64")
    tn.tn_batch_run(b)
    assert rel_err(tn.tn_batch_read(b), ref) < FP64_TOL
    tn.tn_batch_free(b)


def test_full_family_one_launch(tn, family):
    """All 32 circuits x 1024 bitstrings, truncated: one graph launch; the batch equals single
    calls, a replay repeats it bit for bit, new bitstrings run through the same graph, and BF16x6
    stays within 1e-5 of FP64 for nearly every amplitude above round-off."""
    plans = _plans(tn, family)
    chis = [chi for _, _, _, chi in plans]
    assert min(chis) >= 2
    ps = [p for _, _, p, _ in plans]
    bits = [w.bits for w in family]
    b64 = tn.tn_batch_create(ps, [x[:64] for x in bits], "fp64", hbm_budget_bytes=32.0 * 2 ** 30)
    btc = tn.tn_batch_create(ps, bits, "bf16x6", hbm_budget_bytes=32.0 * 2 ** 30)
    info = tn.tn_batch_info(btc)
    assert info["graph_kernels"] >= 32
    assert info["device_bytes"] <= 32.0 * 2 ** 30 + 64 * 2 ** 20     # workspaces within the budget
    tn.tn_launch_count(reset=True)
    tn.tn_batch_run(btc)
    assert tn.tn_launch_count() == info["graph_kernels"]
    a_tc = tn.tn_batch_read(btc)
    tn.tn_batch_run(b64)
    a64 = tn.tn_batch_read(b64)
    # at chi = 2 the truncation leaves round-off-level amplitudes (rms ~1e-17 against 2^-n/2 for
    # the exact ones): precisions are compared on the circuits whose amplitudes lie above that
    checked, within, worst = 0, 0, 0.0
    for g_tc, g64, w in zip(btc.split(a_tc), b64.split(a64), family):
        g_tc = g_tc[:len(g64)]
        rms = np.sqrt(np.mean(np.abs(g64) ** 2))
        if not rms > 1e-8 * 2.0 ** (-w.graph.n / 2):
            continue
        r = np.abs(g_tc - g64) / rms
        checked += len(r)
        within += int(np.sum(r <= TC_TOL))
        worst = max(worst, float(r.max()))
    assert checked >= 64
    assert within >= 0.99 * checked and worst < 1e-4
    for i in (0, 15, 31):
        assert np.array_equal(btc.split(a_tc)[i], tn.tn_amplitudes(ps[i], bits[i], "bf16x6"))
    tn.tn_batch_run(btc)
    assert np.array_equal(tn.tn_batch_read(btc), a_tc)            # a replay is deterministic
    rng = np.random.default_rng(7)
    new = [rng.integers(0, 2, size=(len(w.bits), w.graph.n)) for w in family]
    tn.tn_batch_set_bits(btc, new)
    tn.tn_batch_run(btc)
    got = btc.split(tn.tn_batch_read(btc))
    for i in (0, 15, 31):
        assert np.array_equal(got[i], tn.tn_amplitudes(ps[i], new[i], "bf16x6"))
    tn.tn_batch_free(btc)
    tn.tn_batch_free(b64)


def test_batch_rejects_stale_plan(tn, family):
    w = family[0]
    c, p, chi = tn.tn_build_largest_chi(w.graph.n, w.graph.edges, w.gates, w.split)
    b = tn.tn_batch_create([p], [w.bits[:8]], "fp64")
    tn.tn_evolve_two_sided(c, w.split, chi * 2, 1e-12)        # other arguments: new shapes
    with pytest.raises(tn.TNError) as ei:
        tn.tn_batch_run(b)
    assert ei.value.status == tn.TN_ERR_STATE
    tn.tn_batch_free(b)


@pytest.mark.parametrize("name,n_bits,prec,tol", [
    ("syc53", 512, "bf16x6", TC_TOL),
    ("syc53", 64, "fp64", FP64_TOL),
    ("grid12", 256, "tf32x3", 2e-4),
])
def test_autotune_keeps_results(tn, name, n_bits, prec, tol):
    w = gen.workload(name, n_bits=n_bits)
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff)
    p = tn.tn_path(c)
    before = tn.tn_plan_kernels(p, prec)
    a0 = tn.tn_amplitudes(p, w.bits, prec)
    ref = tn.tn_amplitudes(p, w.bits, "fp64")
    chosen = tn.tn_autotune(p, prec, n_bits)
    assert len(chosen) == p.info["n_steps"] == len(before)
    assert tn.tn_plan_kernels(p, prec) == chosen
    assert all(not k.isdigit() for k in chosen)
    a1 = tn.tn_amplitudes(p, w.bits, prec)
    if prec == "bf16x6":
        # every amplitude within 1e-5 of FP64, with the heuristic's kernels and the tuned ones
        for a in (a0, a1):
            assert rel_err(a, ref) < tol
        assert any(k.startswith("tcgen05") for k in chosen)
    else:
        assert rel_err(a1, ref) < tol
        assert rel_err(a0, ref) < tol


@pytest.mark.parametrize("name,n_bits,opts", [
    ("syc53", 96, {}),
    ("grid20", 2, {"max_intermediate": 1 << 22}),       # slices, ragged K and N tiles
])
def test_tma_built_operand_equals_loaded_operand(tn, name, n_bits, opts):
    """The three ways the TMA-fed BF16x6 step gets its overlap operand (built in shared memory from
    the node tensors, read as complex64 and split on chip, loaded as bf16 pieces from a formation
    pass) give the same values to the same MMAs: identical amplitudes."""
    w = gen.workload(name, n_bits=n_bits)
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff)
    p = tn.tn_path(c, **opts)
    ks = tn.tn_plan_kernels(p, "bf16x6")
    assert "tcgen05_tma" in ks
    results = {}
    modes = ("tcgen05_tma", "tcgen05_tma_buildb", "tcgen05_tma_loadb")
    for mode in modes:
        for bn in ("", "_bn64"):
            forced = [k if not k.startswith("tcgen05_tma") else mode + bn for k in ks]
            tn.tn_plan_set_kernels(p, "bf16x6", forced)
            results[(mode, bn)] = tn.tn_amplitudes(p, w.bits, "bf16x6")
    tn.tn_plan_set_kernels(p, "bf16x6", None)
    for bn in ("", "_bn64"):
        for mode in modes[1:]:
            assert np.array_equal(results[(modes[0], bn)], results[(mode, bn)]), (mode, bn)
    ref = tn.tn_amplitudes(p, w.bits, "fp64")
    tol = TC_TOL
    for v in results.values():
        assert rel_err(v, ref) < tol
    with pytest.raises(tn.TNError):
        tn.tn_plan_set_kernels(p, "bf16x6", ["tcgen05_split"] * p.info["n_steps"])
