"""Serving loop (continuous batching over resident plans): each request's amplitudes are the same
in the mix as alone, admission is by device memory, and waits are bounded."""
import numpy as np
import pytest

import gen
from tests.gpu_common import FP64_TOL, TC_TOL, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2011_02621_gb300 import build
    build.build()
    from paper_2011_02621_gb300 import tn as _tn
    return _tn


def _plan(tn, w, **opts):
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff)
    return tn.tn_path(c, mem_budget_bytes=2 * 2 ** 30, **opts)


def test_mixed_requests_match_alone(tn):
    rng = np.random.default_rng(17)
    w12 = gen.workload("grid12", n_bits=1)
    w53 = gen.workload("syc53", n_bits=1)
    g = gen.random_regular3(16, gen.rng(77, 0))
    gates = gen.rqc(g, 6, gen.rng(77, 1), sequence="".join(sorted(g.patterns)), oneq="haar")
    wr = gen.Workload("reg16", g, gates, 6, 3, 0, 1e-12, gen.bitstrings(16, 1, gen.rng(77, 2)))
    plans = {"grid12": (_plan(tn, w12), 12), "syc53": (_plan(tn, w53), 53), "reg16": (_plan(tn, wr), 16)}
    srv = tn.tn_server_create(hbm_budget_bytes=6 * 2 ** 30, max_inflight=4)
    jobs = []
    for i in range(24):
        name = ["grid12", "syc53", "reg16"][i % 3]
        prec = ["fp64", "bf16x6", "fp32"][(i // 3) % 3]
        p, n = plans[name]
        bits = gen.bitstrings(n, int(rng.integers(1, 300)), gen.rng(500 + i, 2))
        jobs.append((name, prec, bits, tn.tn_server_submit(srv, p, bits, prec)))
    for name, prec, bits, t in jobs:
        got = tn.tn_server_wait(srv, t)
        alone = tn.tn_amplitudes(plans[name][0], bits, prec)
        tol = FP64_TOL if prec == "fp64" else TC_TOL
        assert rel_err(got, alone) < tol, (name, prec)
    st = tn.tn_server_stats_get(srv)
    assert st["completed"] == 24 and st["failed"] == 0
    assert st["p99_latency_s"] >= st["p50_latency_s"] > 0
    assert st["max_inflight_seen"] >= 1 and st["peak_admitted_bytes"] <= 6 * 2 ** 30
    tn.tn_server_free(srv)


def test_admission_refuses_requests_beyond_budget(tn):
    w = gen.workload("syc53", n_bits=64)
    p = _plan(tn, w)
    srv = tn.tn_server_create(hbm_budget_bytes=1e6, max_inflight=2)
    with pytest.raises(tn.TNError) as ei:
        tn.tn_server_submit(srv, p, w.bits, "fp64")
    assert ei.value.status == tn.TN_ERR_OOM
    assert tn.tn_server_stats_get(srv)["rejected"] == 1
    tn.tn_server_free(srv)


def test_bounded_wait_and_bad_request(tn):
    w = gen.workload("syc53", n_bits=1024)
    p = _plan(tn, w)
    srv = tn.tn_server_create(max_inflight=1)
    t = tn.tn_server_submit(srv, p, w.bits, "fp64")          # ~2 s of FP64 work
    with pytest.raises(tn.TNError) as ei:
        tn.tn_server_wait(srv, t, timeout_ms=0)
    assert ei.value.status == tn.TN_ERR_TIMEOUT
    a = tn.tn_server_wait(srv, t)                            # then completes
    assert a.shape == (1024,) and np.all(np.isfinite(a))
    with pytest.raises(tn.TNError) as ei:
        tn._check(tn.LIB.tn_server_submit(srv.ptr, p.ptr, None, 5, 0, None, None))
    assert ei.value.status == tn.TN_ERR_ARG
    tn.tn_server_free(srv)
