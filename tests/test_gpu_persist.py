"""The persistent TMA-fed tcgen05 step (one CTA per SM walking the output tiles) through the C ABI.

Where it keeps the accumulators of the one-tile-per-CTA step (128-column tiles, K > 64: three
order-0 accumulators, one set) it issues the same MMAs and sums them in the same order, so the
amplitudes must be bit-identical to that kernel's (the 4x5 grid cut into slices has such steps).
At 128-column tiles with K <= 64 it keeps one order-0 accumulator and two accumulator sets, and at
64-column tiles three order-0 accumulators where the other kernel keeps seven; there the
amplitudes are held to the tensor-core bound (1e-5 relative to rms|a|) against the FP64 path and
the brute-force state vector. The form that reads its input as complex64 and splits it on chip
makes the pieces the previous step would have written, so it is bit-identical to the form that
loads them. Each persistent CTA walks many tiles in the large-batch cases."""
import numpy as np
import pytest

import gen
from oracle import statevector as sv
from tests.gpu_common import TC_TOL, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2011_02621_gb300 import build
    build.build()
    from paper_2011_02621_gb300 import tn as _tn
    return _tn


def supported(tn, p, kernel):
    """Indices of the steps that accept `kernel` (each tried alone on the heuristic list)."""
    base = tn.tn_plan_kernels(p, "bf16x6")
    ok = []
    for i in range(len(base)):
        trial = list(base)
        trial[i] = kernel
        try:
            tn.tn_plan_set_kernels(p, "bf16x6", trial)
            ok.append(i)
        except Exception:
            pass
    tn.tn_plan_set_kernels(p, "bf16x6", None)
    return base, ok


def run_with(tn, p, bits, base, steps, kernel):
    ks = list(base)
    for i in steps:
        ks[i] = kernel
    tn.tn_plan_set_kernels(p, "bf16x6", ks)
    tn.tn_profile_enable(True)
    a = tn.tn_amplitudes(p, bits, "bf16x6")
    prof = tn.tn_profile_read()
    tn.tn_profile_enable(False)
    tn.tn_plan_set_kernels(p, "bf16x6", None)
    return a, prof


def persistent_launches(prof):
    return sum(v["launches"] for k, v in prof.items() if k.startswith("contract_step_tcgen05_tma_persist"))


def launched_on_every_step(prof, steps):
    """The persistent kernel ran once per chosen step in every batch chunk."""
    n = persistent_launches(prof)
    return n > 0 and n % len(steps) == 0


def syc53_plan(tn, layers):
    w = gen.workload("syc53", n_bits=256)
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff)
    return w, c, tn.tn_path(c, layers=layers, mem_budget_bytes=32 * 2 ** 30)


@pytest.fixture(scope="module")
def grid20_cut(tn):
    """The 4x5 grid at 14 cycles on its double-layer plan cut into 128 slices (several (bitstring,
    slice) items per bitstring, ragged tiles, K up to 128)."""
    w = gen.workload("grid20", n_bits=16)
    ref = sv.amplitudes(sv.run(20, w.gates), w.bits)
    c = tn.tn_build(20, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split)
    p = tn.tn_path(c, layers=2, max_intermediate=1 << 20)
    assert p.info["n_slices"] > 1
    return w, ref, c, p


@pytest.mark.parametrize("layers", [2, 1])
def test_bn128_on_syc53_vs_fp64(tn, layers):
    w, c, p = syc53_plan(tn, layers)
    base, ok = supported(tn, p, "tcgen05_tma_persist_bn128")
    assert ok, "no step takes the 128-column persistent kernel"
    a2, prof = run_with(tn, p, w.bits, base, ok, "tcgen05_tma_persist_bn128")
    assert launched_on_every_step(prof, ok)
    a64 = tn.tn_amplitudes(p, w.bits[:64], "fp64")
    assert rel_err(a2[:64], a64) < TC_TOL
    a1, _ = run_with(tn, p, w.bits, base, ok, "tcgen05_tma_bn128")
    assert rel_err(a2, a1) < TC_TOL


@pytest.mark.parametrize("opts", [{"layers": 2, "max_intermediate": 1 << 20}, {"layers": 2},
                                  {"layers": 1, "max_intermediate": 1 << 22}])
def test_long_k_bit_identical_to_one_tile_per_cta(tn, opts):
    """Steps with 64 < K < 256 on 128-column tiles of the 4x5 grid plans: the same accumulators,
    the same bits."""
    w = gen.workload("grid20", n_bits=4)
    c = tn.tn_build(20, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split)
    p = tn.tn_path(c, mem_budget_bytes=16 * 2 ** 30, **opts)
    _, _, mkn = tn.tn_plan_details(p)
    base, ok = supported(tn, p, "tcgen05_tma_persist_bn128")
    long_k = [i for i in ok if mkn[i][1] > 64]
    if not long_k:
        pytest.skip("no long-K step on 128-column tiles: " + str([tuple(int(x) for x in mkn[i]) for i in ok]))
    a1, _ = run_with(tn, p, w.bits, base, long_k, "tcgen05_tma_bn128")
    a2, prof = run_with(tn, p, w.bits, base, long_k, "tcgen05_tma_persist_bn128")
    assert launched_on_every_step(prof, long_k)
    assert np.array_equal(a1, a2)
    ref = sv.amplitudes(sv.run(20, w.gates), w.bits)
    assert rel_err(a2, ref) < TC_TOL


def test_large_batch_vs_fp64(tn):
    """16384 bitstrings: every persistent CTA walks hundreds of tiles through its operand ring."""
    w, c, p = syc53_plan(tn, 2)
    bits = gen.bitstrings(w.graph.n, 16384, gen.rng(11, 3))
    pick = np.concatenate([np.arange(32), 8192 + np.arange(32), 16384 - 32 + np.arange(32)])
    a64 = tn.tn_amplitudes(p, bits[pick], "fp64")
    for kernel in ("tcgen05_tma_persist", "tcgen05_persist_c64"):
        base, ok = supported(tn, p, kernel)
        a2, prof = run_with(tn, p, bits, base, ok, kernel)
        assert launched_on_every_step(prof, ok), kernel
        assert np.all(np.isfinite(a2)), kernel
        assert rel_err(a2[pick], a64) < TC_TOL, kernel


PERSIST_FORMS = ["tcgen05_tma_persist", "tcgen05_persist_c64", "tcgen05_persist_loadb", "tcgen05_persist_c64_loadb"]


@pytest.mark.parametrize("kernel", [f + w for f in PERSIST_FORMS for w in ("", "_bn128", "_bn64")])
def test_grid20_cut_plan_vs_statevector(tn, grid20_cut, kernel):
    w, ref, c, p = grid20_cut
    base, ok = supported(tn, p, kernel)
    assert ok, kernel
    a2, prof = run_with(tn, p, w.bits, base, ok, kernel)
    assert launched_on_every_step(prof, ok), kernel
    assert rel_err(a2, ref) < TC_TOL, kernel


def test_bn64_on_syc53_double_layer_vs_fp64(tn):
    w, c, p = syc53_plan(tn, 2)
    base, ok = supported(tn, p, "tcgen05_tma_persist_bn64")
    assert ok
    a2, prof = run_with(tn, p, w.bits, base, ok, "tcgen05_tma_persist_bn64")
    assert launched_on_every_step(prof, ok)
    a64 = tn.tn_amplitudes(p, w.bits, "fp64")
    assert rel_err(a2, a64) < TC_TOL


@pytest.mark.parametrize("width", ["_bn128", "_bn64"])
@pytest.mark.parametrize("plan", ["syc53_double_layer", "syc53_overlap", "grid20_cut"])
def test_operand_forms_bit_identical(tn, grid20_cut, plan, width):
    """The four forms of the persistent kernel make the same bf16 pieces in shared memory: the
    input as the pieces its producer wrote (TMA) or as complex64 split on chip, the overlap operand
    as complex64 split on chip or as pieces formed in HBM (once per slice for a ket tensor) and
    loaded by TMA. So their amplitudes agree bit for bit (the previous step writes complex64 in one
    case, pieces in the other)."""
    if plan == "grid20_cut":
        w, _, c, p = grid20_cut
        bits = w.bits
    else:
        w, c, p = syc53_plan(tn, 2 if plan == "syc53_double_layer" else 1)
        bits = w.bits if plan == "syc53_overlap" else gen.bitstrings(w.graph.n, 4096, gen.rng(11, 5))
    base, ok = supported(tn, p, PERSIST_FORMS[0] + width)
    if not ok:
        pytest.skip("no step of this plan takes the kernel at this width")
    a1, _ = run_with(tn, p, bits, base, ok, PERSIST_FORMS[0] + width)
    assert np.all(np.isfinite(a1))
    for form in PERSIST_FORMS[1:]:
        _, ok2 = supported(tn, p, form + width)
        assert ok == ok2, form
        a2, prof = run_with(tn, p, bits, base, ok, form + width)
        assert launched_on_every_step(prof, ok), form
        assert np.array_equal(a1, a2), form


def test_autotuner_result_on_syc53_double_layer_vs_fp64(tn):
    """The tuner may pick the persistent kernels, and charges a kernel that reads bf16 pieces the
    cost of the pieces its producer writes; whatever it picks stays within the bound."""
    w, c, p = syc53_plan(tn, 2)
    ks = tn.tn_autotune(p, "bf16x6", len(w.bits))
    assert len(ks) == p.info["n_steps"]
    a = tn.tn_amplitudes(p, w.bits, "bf16x6")
    a64 = tn.tn_amplitudes(p, w.bits, "fp64")
    assert rel_err(a, a64) < TC_TOL
