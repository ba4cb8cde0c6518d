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


def test_device_memory_stays_within_the_budget(tn):
    """Several plans and workers: every worker's workspace lives only as long as its batch, so the
    device memory the allocator hands out while the server runs (PyTorch's peak over its baseline)
    stays within the admission budget (plus the allocator's rounding of each block)."""
    import torch
    plans = []
    for name, opts in (("grid12", {}), ("syc53", {}), ("syc53", {"layers": 2})):
        w = gen.workload(name, n_bits=1)
        plans.append((_plan(tn, w, **opts), w.graph.n))
    budget = 2.5 * 2 ** 30                  # above any one request (plans hold 2 GiB batches), below several
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    srv = tn.tn_server_create(hbm_budget_bytes=budget, max_inflight=3)
    tickets = []
    for i in range(18):
        p, n = plans[i % 3]
        bits = gen.bitstrings(n, 200 + 37 * i, gen.rng(900 + i, 2))
        tickets.append(tn.tn_server_submit(srv, p, bits, ["bf16x6", "fp32", "fp64"][i % 3]))
    for t in tickets:
        tn.tn_server_wait(srv, t)
    st = tn.tn_server_stats_get(srv)
    tn.tn_server_free(srv)
    torch.cuda.synchronize()
    assert st["completed"] == 18 and st["peak_admitted_bytes"] <= budget
    peak = torch.cuda.max_memory_allocated() - base
    assert peak <= 1.05 * budget + 64 * 2 ** 20, (peak, budget)
    assert torch.cuda.memory_allocated() <= base + 2 * 2 ** 20   # nothing kept after the server


def test_queued_requests_can_be_cancelled(tn):
    """One worker busy with a large batch; requests queued behind it are cancelled on the host:
    they are removed, never run, and their tickets are forgotten; the others complete as alone."""
    w = gen.workload("syc53", n_bits=1)
    p = _plan(tn, w, layers=2)
    srv = tn.tn_server_create(hbm_budget_bytes=8 * 2 ** 30, max_inflight=1)
    big = tn.tn_server_submit(srv, p, gen.bitstrings(53, 16384, gen.rng(31, 2)), "fp64")
    keep_bits = gen.bitstrings(53, 40, gen.rng(32, 2))
    keep = tn.tn_server_submit(srv, p, keep_bits, "fp32")
    drop = [tn.tn_server_submit(srv, p, gen.bitstrings(53, 50, gen.rng(33 + i, 2)), "fp32") for i in range(3)]
    for t in drop:
        tn.tn_server_cancel(srv, t)
    with pytest.raises(tn.TNError) as ei:
        tn.tn_server_cancel(srv, drop[0])              # already gone
    assert ei.value.status == tn.TN_ERR_ARG
    got = tn.tn_server_wait(srv, keep)
    tn.tn_server_wait(srv, big)
    with pytest.raises(tn.TNError) as ei:
        tn.tn_server_cancel(srv, keep)                 # complete (and collected): unknown now
    assert ei.value.status == tn.TN_ERR_ARG
    with pytest.raises(tn.TNError) as ei:
        tn.tn_server_wait(srv, drop[1])
    assert ei.value.status == tn.TN_ERR_ARG
    st = tn.tn_server_stats_get(srv)
    assert st["cancelled"] == 3 and st["completed"] == 2 and st["amplitudes"] == 16384 + 40
    assert rel_err(got, tn.tn_amplitudes(p, keep_bits, "fp32")) < TC_TOL
    tn.tn_server_free(srv)


def test_running_request_cannot_be_cancelled(tn):
    w = gen.workload("syc53", n_bits=1)
    p = _plan(tn, w, layers=2)
    srv = tn.tn_server_create(hbm_budget_bytes=8 * 2 ** 30, max_inflight=1)
    t = tn.tn_server_submit(srv, p, gen.bitstrings(53, 16384, gen.rng(41, 2)), "fp64")
    import time
    for _ in range(200):                               # until the worker has taken it
        st = tn.tn_server_stats_get(srv)
        if st["max_inflight_seen"] >= 1:
            break
        time.sleep(0.005)
    with pytest.raises(tn.TNError) as ei:
        tn.tn_server_cancel(srv, t)
    assert ei.value.status == tn.TN_ERR_STATE
    tn.tn_server_wait(srv, t)
    tn.tn_server_free(srv)
