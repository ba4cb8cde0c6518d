"""Bounded device loops end with an error status, not a hang, and leave the context usable.

The one-sided Jacobi SVD of every compression (Eqs. svd/svd2) runs at most a capped number of
sweeps (tn_set_svd_sweeps; the default 60). With a cap of one sweep, matrices that need more end
unconverged: the kernel sets its error word, the call returns TN_ERR_TIMEOUT, and with the cap
lifted the same circuit and plan give the right amplitudes again."""
import pytest

import gen
from oracle import statevector as sv
from tests.gpu_common import FP64_TOL, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2011_02621_gb300 import build
    build.build()
    from paper_2011_02621_gb300 import tn as _tn
    return _tn


def test_sweep_cap_on_the_ket_half(tn):
    w = gen.workload("grid12", n_bits=16)
    c = tn.tn_build(12, w.graph.edges, w.gates)
    tn.tn_set_svd_sweeps(c, 1)
    with pytest.raises(tn.TNError) as ei:
        tn.tn_evolve_two_sided(c, w.split)
    assert ei.value.status == tn.TN_ERR_TIMEOUT and "sweep" in str(ei.value)
    tn.tn_set_svd_sweeps(c, 0)
    tn.tn_evolve_two_sided(c, w.split)
    ref = sv.amplitudes(sv.run(12, w.gates), w.bits)
    assert rel_err(tn.tn_amplitudes(tn.tn_path(c), w.bits, "fp64"), ref) < FP64_TOL


def test_sweep_cap_on_the_bra_half(tn):
    w = gen.workload("grid12", n_bits=16)
    c = tn.tn_build(12, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split)
    p = tn.tn_path(c)
    ref = sv.amplitudes(sv.run(12, w.gates), w.bits)
    tn.tn_set_svd_sweeps(c, 1)                        # the bra program of later amplitude calls
    for prec in ("fp64", "fp32"):
        with pytest.raises(tn.TNError) as ei:
            tn.tn_amplitudes(p, w.bits, prec)
        assert ei.value.status == tn.TN_ERR_TIMEOUT and "bra half" in str(ei.value)
    tn.tn_set_svd_sweeps(c, 0)
    assert rel_err(tn.tn_amplitudes(p, w.bits, "fp64"), ref) < FP64_TOL
    with pytest.raises(tn.TNError) as ei:
        tn.tn_set_svd_sweeps(c, -1)
    assert ei.value.status == tn.TN_ERR_ARG
