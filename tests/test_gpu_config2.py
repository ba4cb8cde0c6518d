"""The precision workload at its stated size: the 4x5 grid at 14 cycles (untruncated), 4096 seeded
bitstrings per precision form through the C ABI on the joined double-layer plan, each form
element by element against the 2^20 state vector, FP64 on 256 of them, and 16 against the oracle's
stored amplitudes (tests/golden/grid20_oracle.json).

Bounds: 1e-5 relative to rms |a| for FP32 and the tensor-core forms that carry about 24-bit
products (BF16x6, TF32x3, TF32x6); BF16x3 (hi/lo bf16 pieces, about 16-bit products) 1e-4; single
TF32 (10-bit mantissa) 1e-2; FP64 1e-10."""
import json
import os

import numpy as np
import pytest

import gen
from oracle import statevector as sv
from tests.gpu_common import FP64_TOL, TC_TOL, rel_err

pytestmark = pytest.mark.gpu

BOUND = {"fp32": TC_TOL, "bf16x6": TC_TOL, "tf32x3": TC_TOL, "tf32x6": TC_TOL, "bf16x3": 1e-4, "tf32": 1e-2}
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "grid20_oracle.json")


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2011_02621_gb300 import build
    build.build()
    from paper_2011_02621_gb300 import tn as _tn
    return _tn


@pytest.fixture(scope="module")
def grid20(tn):
    w = gen.workload("grid20")
    assert len(w.bits) == 4096
    ref = sv.amplitudes(sv.run(20, w.gates), w.bits)
    c = tn.tn_build(20, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split)
    p = tn.tn_path(c, layers=2, mem_budget_bytes=64 * 2 ** 30)
    return w, ref, c, p


@pytest.mark.parametrize("prec", ["fp32", "bf16x6", "tf32x3", "tf32x6", "bf16x3", "tf32"])
def test_every_form_on_4096_bitstrings_vs_statevector(tn, grid20, prec):
    w, ref, c, p = grid20
    tn.tn_profile_enable(True)
    a = tn.tn_amplitudes(p, w.bits, prec)
    prof = tn.tn_profile_read()
    tn.tn_profile_enable(False)
    if prec != "fp32":
        assert sum(v["launches"] for k, v in prof.items() if "tcgen05" in k) > 0, prec
    assert rel_err(a, ref) < BOUND[prec], (prec, rel_err(a, ref))


def test_fp64_and_the_oracle(tn, grid20):
    w, ref, c, p = grid20
    a64 = tn.tn_amplitudes(p, w.bits[:256], "fp64")
    assert rel_err(a64, ref[:256]) < FP64_TOL
    d = json.load(open(GOLDEN))
    bits = np.array(d["bits"], dtype=np.uint8)
    assert np.array_equal(bits, w.bits[:len(bits)])
    ora = np.array([complex(r, i) for r, i in d["amplitudes"]])
    assert rel_err(a64[:len(ora)], ora) < FP64_TOL
    assert rel_err(tn.tn_amplitudes(p, bits, "bf16x6"), ora) < TC_TOL
