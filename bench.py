#!/usr/bin/env python
"""Benchmark of the TNS amplitude path on one GB300 per rank.

Workload (one "step"): the 53-qubit staggered diagonal-coupled grid (6 rows x
9 columns minus one seeded site), 10 cycles ABCDCDABAB, two-sided evolution
split after cycle 5, bonds truncated to chi = 64 or singular values below
1e-8 s_0; one step = the ket evolution + the batched bra evolution and the
path-ordered contraction of the double-layer network (joined partial paths)
with the FP64 slice sum, for 65536 seeded random bitstrings. Synthetic seeded inputs stand in for the Sycamore layout and
circuits, which are not available.

Prints ONE JSON line (rank 0). ``--impl reference`` times the CPU oracle
instead (the reference arm of this benchmark).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "amplitudes/s @ rel.err≤1e-5 vs FP64 (53q d10); contraction TFLOP/s; p99 latency"
UNIT = "amplitudes/s"
WORKLOAD = ("53-qubit staggered grid (6x9 minus 1 seeded site), 10 cycles ABCDCDABAB, split 5, chi 64, "
            "cutoff 1e-8, 65536 random bitstrings per step")
TOL = 1e-5
NOMINAL = {"tf32_over_bf16": 1.1 / 2.25, "fp32_simt_tflops": 152 * 128 * 2 * 2.07e9 / 1e12,
           "fp64_tflops": 1.25}


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=float(d["hbm_gbs"]), bf16_tflops=float(d["bf16_tflops"]),
                    bf16_tflops_sustained=float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), source="measured")
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, source="fallback")


# ---------------------------------------------------------------------------
# CPU oracle leg (also the reference arm)
# ---------------------------------------------------------------------------
def _oracle_worker(payload):
    """Runs in a spawned process with single-threaded BLAS: oracle amplitudes for a few bitstrings."""
    import numpy as np  # noqa: F401
    import gen
    from oracle import tns
    name, idx, n_bits, seed_off, compress = payload
    w = gen.workload(name, n_bits=n_bits)
    bits = _rank_bits(w, seed_off)[list(idx)]
    g1, g2 = tns.split_gates(w.gates, w.split)
    ket = tns.evolve_ket(w.graph.n, w.graph.edges, g1, w.chi, w.cutoff, compress)
    t0 = time.perf_counter()
    a, _ = tns.amplitudes(w.graph.n, w.graph.edges, w.gates, bits, w.split, w.chi, w.cutoff, ket=ket,
                          compress=compress)
    return list(idx), [complex(x) for x in a], time.perf_counter() - t0


def _rank_bits(w, seed_off):
    import gen
    if seed_off == 0:
        return w.bits
    return gen.bitstrings(w.graph.n, len(w.bits), gen.rng(gen.BASE_SEED + 3 + 7919 * seed_off, 2))


def cpu_oracle(name, n_bits, sample, seed_off=0, cores=None, compress="one_sided"):
    """Time the oracle (as it stands) on `sample` bitstrings over a spawned process pool
    (compress: the bond compression of both halves, as in the oracle)."""
    import multiprocessing as mp
    import numpy as np
    cores = cores or os.cpu_count() or 1
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    per = max(1, math.ceil(sample / cores))
    chunks = [(name, tuple(range(i, min(i + per, sample))), n_bits, seed_off, compress)
              for i in range(0, sample, per)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(cores, len(chunks))) as pool:
        pool.map(_oracle_worker, [(name, (0,), n_bits, seed_off, compress)] * min(cores, len(chunks)))   # warm imports
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, chunks)
        wall = time.perf_counter() - t0
    amps = np.zeros(sample, dtype=np.complex128)
    busy = 0.0
    for idx, a, dt in res:
        amps[list(idx)] = a
        busy += dt
    return dict(value=sample / wall, single_thread_value=sample / busy, cores=min(cores, len(chunks)),
                wall_s=wall, cpu_s=busy, amps=amps)


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    sample = args.ref_sample
    vals = []
    for _ in range(args.warmup):
        cpu_oracle("syc53", args.bits, max(2, sample // 8))
    t_all = 0.0
    for _ in range(args.steps):
        r = cpu_oracle("syc53", args.bits, sample)
        vals.append(r)
        t_all += r["wall_s"]
    value = sum(r["value"] for r in vals) / len(vals)
    cores = vals[0]["cores"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * t_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} of the workload's bitstrings per step (ket evolution outside)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def traffic_record(kind, network="double_layer"):
    """DRAM bytes of `kind` on `network`'s plan relative to its algorithmic bytes, from a committed
    ncu capture of a small case (profiles/traffic.json), if the kernel sources are unchanged since
    the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    rec = d.get(network, {}).get(kind)
    if not rec or rec.get("source_sha") != source_sha(kind):
        return None
    return rec


# the sources of each kernel kind with a traffic record (kernel and headers)
_BOX = ("stream.cu", "tn_device.h", "tn_internal.h", "tn_smem.h")
TRAFFIC_SOURCES = {"contract_step_tcgen05_tma": ("tc_tma.cu", "tn_device.h", "tn_internal.h"),
                   "contract_step_fp32_box": _BOX, "contract_step_fp32_box_tc_fallback": _BOX,
                   "gate_svd_fp64": ("evolve.cu", "tn_internal.h", "tn_smem.h")}


def source_sha(kind="contract_step_tcgen05_tma"):
    """Hash of a kernel kind's sources: a traffic record taken on other sources is stale."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2011_02621_gb300", "csrc")
    for f in TRAFFIC_SOURCES.get(kind, TRAFFIC_SOURCES["contract_step_tcgen05_tma"]):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------
# serving: a seeded Poisson request stream over three circuit classes
# ---------------------------------------------------------------------------
# (workload, size cap): the 104-qubit class is capped at 64 bitstrings per request so that the plain
# FP64 form (about 30 ms of FP64 contraction per 104-qubit amplitude) serves the same stream
SERVE_CLASSES = (("syc104", 64), ("syc53", 65536), ("grid20", 16))


def batch_run(tn, np, torch, prec, steps, warmup, flush, depth=12, truncated=True):
    """32 circuits on random 3-regular graphs (24..40 qubits), 1024 bitstrings each, as one graph
    launch; beside it the same work as 32 sequential tn_amplitudes calls, and end to end with host
    copies. truncated: each circuit at the largest chi with no cut at 2^24 elements (its amplitudes
    have no exact reference; at chi = 2 they are round-off level, so the FP64 comparison covers
    the circuits above that); else untruncated (exact amplitudes, counted within 1e-5 of FP64)."""
    import gen
    fam = gen.regular3_family(count=32, depth=depth, n_bits=1024)
    stream = torch.cuda.current_stream()
    plans, chis, cmacs = [], [], 0.0
    for w in fam:
        if truncated:
            c, p, chi = tn.tn_build_largest_chi(w.graph.n, w.graph.edges, w.gates, w.split)
        else:
            c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
            tn.tn_evolve_two_sided(c, w.split)
            p, chi = tn.tn_path(c), 0
        tn.tn_autotune(p, prec, len(w.bits), stream=stream)
        plans.append(p)
        chis.append(chi)
        cmacs += p.info["cmacs"] * len(w.bits)
    bits = [w.bits for w in fam]
    b = tn.tn_batch_create(plans, bits, prec, hbm_budget_bytes=48.0 * 2 ** 30, stream=stream)
    # FP64 reference on the first 64 bitstrings of every circuit
    b64 = tn.tn_batch_create(plans, [x[:64] for x in bits], "fp64", hbm_budget_bytes=48.0 * 2 ** 30, stream=stream)
    total = b.total

    def timed(fn):
        for _ in range(warmup):
            fn()
        t = 0.0
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            t += e0.elapsed_time(e1) / 1000.0
        return t / steps

    t_graph = timed(lambda: tn.tn_batch_run(b, stream=stream))
    a_tc = tn.tn_batch_read(b, stream=stream)
    tn.tn_batch_run(b64, stream=stream)
    a64 = tn.tn_batch_read(b64, stream=stream)
    checked = ok = 0
    worst = 0.0
    for g, r, w in zip(b.split(a_tc), b64.split(a64), fam):
        g = g[:len(r)]
        rms = float(np.sqrt(np.mean(np.abs(r) ** 2)))
        if not rms > 1e-8 * 2.0 ** (-w.graph.n / 2):
            continue                    # round-off-level amplitudes: no meaningful comparison
        e = np.abs(g - r) / rms
        checked += len(e)
        ok += int(np.sum(e <= TOL))
        worst = max(worst, float(e.max()))
    frac = ok / max(checked, 1)
    dev_bits = [torch.from_numpy(tn.pack_bits(x).view(np.int64).copy()).cuda() for x in bits]
    dev_out = [torch.empty(len(x), dtype=torch.complex128, device="cuda") for x in bits]

    def sequential():
        for p, x, o in zip(plans, dev_bits, dev_out):
            tn.tn_amplitudes(p, x, prec, out=o, stream=stream)

    t_seq = timed(sequential)
    flat, _ = tn._packed_concat(plans, bits)
    pin_bits = torch.from_numpy(flat.view(np.int64).copy()).pin_memory()
    pin_out = torch.empty(total, dtype=torch.complex128).pin_memory()

    def e2e():
        tn.tn_batch_set_bits(b, pin_bits, stream=stream)
        tn.tn_batch_run(b, stream=stream)
        tn.tn_batch_read(b, out=pin_out, stream=stream)

    t_e2e = timed(e2e)
    info = tn.tn_batch_info(b)
    scale = 1.0 if truncated else frac      # exact amplitudes: count those within 1e-5 of FP64
    res = r3({"workload": f"32 random 3-regular circuits, 24-40 q, {depth} cycles, 1024 bits each"
                          + (", largest chi without cuts" if truncated else ", untruncated"),
              "value": total / t_graph * scale, "ms_per_launch": 1000 * t_graph, "graph_kernels": info["graph_kernels"],
              "vs_fp64": {"compared": checked, "within_1e-5": frac, "max_rel_err": worst},
              "chi_counts": {str(x): chis.count(x) for x in sorted(set(chis))} if truncated else None,
              "sequential_calls_value": total / t_seq * scale,
              "e2e": {"value": total / t_e2e * scale, "h2d_bytes_per_step": int(flat.nbytes),
                      "d2h_bytes_per_step": int(total * 16)}})
    tn.tn_batch_free(b)
    tn.tn_batch_free(b64)
    return res


def serving_run(tn, np, prec, seconds, load=0.8, seed=2011_02621 + 5, plans=None):
    """Replay a Poisson stream of amplitude requests against tn_server_* at `load` times the form's
    measured capacity; sizes log-uniform in [1, cap] per class, classes in equal proportion."""
    import gen
    import time as _t
    if plans is None:
        plans = {}
        for name, cap in SERVE_CLASSES:
            w = gen.workload(name, n_bits=1)
            c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
            tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff)
            plans[name] = (tn.tn_path(c, layers=2, mem_budget_bytes=8.0 * 2 ** 30), w.graph.n, cap)
    # capacity (amplitudes/s) per class in this form, from one batch each
    capacity = {}
    for name, (p, nq, cap) in plans.items():
        nb = max(4, min(cap, 1024 if name != "grid20" else 8))
        bits = gen.bitstrings(nq, nb, gen.rng(seed, 9))
        if prec != "fp64":            # the plain FP64 form keeps the shape heuristic's kernels
            tn.tn_autotune(p, prec, nb)
        tn.tn_amplitudes(p, bits, prec)
        t0 = _t.perf_counter()
        tn.tn_amplitudes(p, bits, prec)
        capacity[name] = nb / (_t.perf_counter() - t0)
    rng = np.random.default_rng(seed)
    names = [n for n, _ in SERVE_CLASSES]
    # expected service seconds per request, mixed over classes; arrival rate for the target load
    mean_size = {n: (cap - 1) / np.log(cap) if cap > 1 else 1.0 for n, cap in SERVE_CLASSES}
    e_service = np.mean([mean_size[n] / capacity[n] for n in names])
    lam = load / e_service
    arrivals, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / lam)
        if t > seconds:
            break
        name = names[int(rng.integers(len(names)))]
        cap = dict(SERVE_CLASSES)[name]
        size = int(np.clip(np.exp(rng.uniform(0, np.log(cap))), 1, cap))
        arrivals.append((t, name, size))
    srv = tn.tn_server_create(hbm_budget_bytes=48.0 * 2 ** 30, max_inflight=4)
    tickets = []
    start = _t.perf_counter()
    for (ta, name, size) in arrivals:
        now = _t.perf_counter() - start
        if ta > now:
            _t.sleep(ta - now)
        p, nq, _ = plans[name]
        bits = gen.bitstrings(nq, size, gen.rng(seed + len(tickets), 2))
        tickets.append((name, size, tn.tn_server_submit(srv, p, bits, prec)))
    for name, size, tk in tickets:
        tn.tn_server_wait(srv, tk)
    wall = _t.perf_counter() - start
    st = tn.tn_server_stats_get(srv)
    tn.tn_server_free(srv)
    return plans, r3({"requests": len(tickets), "amplitudes_per_s": st["amplitudes"] / wall,
                      "p50_latency_s": st["p50_latency_s"], "p99_latency_s": st["p99_latency_s"],
                      "arrival_rate_per_s": lam, "max_inflight_seen": st["max_inflight_seen"]})


def roofline(prof, steps, prec, pk, n_bits, network="double_layer"):
    """The roofline object of the dominant kernel kind of a profiled run: which roof binds it
    (tensor pipe for tcgen05, plain ALU for SIMT FP32 / FP64, else HBM, by its algorithmic
    intensity against the ridge of its compute roof), achieved against that peak, and the DRAM
    traffic of a committed capture when the kernel's sources are unchanged since."""
    kind, rec = max(prof.items(), key=lambda kv: kv[1]["ms"])
    per_launch_s = rec["ms"] / 1000.0 / max(rec["launches"], 1)
    bytes_pl = rec["bytes"] / max(rec["launches"], 1)
    flops_pl = rec["flops"] / max(rec["launches"], 1)
    if "tcgen05" in kind:
        mult = {"tf32x3": 3.0, "bf16x3": 3.0, "bf16x6": 6.0, "tf32x6": 6.0}.get(prec, 1.0)
        if prec.startswith("bf16"):
            c_peak, c_kind = pk["bf16_tflops_sustained"] / mult, "tensor"
        else:
            c_peak, c_kind = pk["bf16_tflops_sustained"] * NOMINAL["tf32_over_bf16"] / mult, "tensor"
    elif "fp64" in kind:
        c_peak, c_kind = NOMINAL["fp64_tflops"], "alu"
    else:
        c_peak, c_kind = NOMINAL["fp32_simt_tflops"], "alu"
    ridge = c_peak * 1e12 / (pk["hbm_gbs"] * 1e9)
    if flops_pl / max(bytes_pl, 1.0) > ridge:
        roof = {"bound": c_kind, "achieved": flops_pl / per_launch_s / 1e12, "peak": c_peak, "unit": "TFLOP/s"}
    else:
        roof = {"bound": "hbm", "achieved": bytes_pl / per_launch_s / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    tr = traffic_record(kind, network)
    # per launch: the captured kernel's DRAM bytes per algorithmic byte times this run's algorithmic
    # bytes per launch (the capture runs a small case whose steps and batch differ from this run's)
    roof["traffic"] = tr["dram_over_algorithmic"] * bytes_pl if tr else None
    roof.update({"kernel": kind, "launches_per_step": rec["launches"] / steps,
                 "algorithmic_bytes_per_launch": bytes_pl, "algorithmic_flops_per_launch": flops_pl,
                 "avg_launch_ms": per_launch_s * 1000,
                 "peak_source": ("measured bf16 sustained x nominal tf32/bf16 ratio, / products per MAC"
                                 if roof["bound"] == "tensor" else
                                 "nominal unit count x 2070 MHz" if roof["bound"] == "alu" else "measured hbm_gbs")
                                + f" ({pk['source']})"})
    return roof


def timed_section(torch, stream, step, steps, warmup, flush):
    """`warmup` untimed calls of step(), then `steps` calls, each after writing the L2-sized flush
    buffer, timed with CUDA events on `stream`; returns the total seconds of the timed calls."""
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1) / 1000.0
    return total


def r3(x):
    """Three significant digits (compact JSON)."""
    if x is None or isinstance(x, (str, bool)):
        return x
    if isinstance(x, dict):
        return {k: r3(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [r3(v) for v in x]
    if isinstance(x, int):
        return x
    return float(f"{x:.3g}")


def top_kernels(prof, steps, k=4):
    """The k kernel kinds with the most device time: ms per step."""
    items = sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:k]
    return {name: r3(v["ms"] / steps) for name, v in items}


def form_run(tn, np, torch, c, w, p, bits_dev, out, prec, steps, warmup, flush, tune=True):
    """One form on plan p: autotuned step kernels, then `steps` timed steps (ket evolution +
    amplitudes of every bitstring in bits_dev, L2 flushed between steps). Returns (seconds per
    step, profile, launches per step, amplitudes on the device)."""
    stream = torch.cuda.current_stream()
    B = len(bits_dev)
    if tune:
        tn.tn_autotune(p, prec, B, stream=stream)

    def step():
        tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff, stream)
        tn.tn_amplitudes(p, bits_dev, prec, out=out, stream=stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    tn.tn_launch_count(reset=True)
    tn.tn_profile_enable(True)
    total = timed_section(torch, stream, step, steps, 0, flush)
    prof = tn.tn_profile_read()
    tn.tn_profile_enable(False)
    return total / steps, prof, tn.tn_launch_count() // steps


def two_sided_run(tn, np, torch, w, packed, idx, a64, prec, steps, warmup, flush, mem_gib, pk):
    """The two-sided bond compression (the singular values of the local product of a gate's two
    endpoints, a variant of Eqs. svd/svd2 the paper does not use) on the device:
    (1) the same workload with both halves compressed two-sided, on the joined double-layer plan:
        FP64 on the bitstrings idx against the one-sided FP64 amplitudes a64 (the cutoff cuts only
        numerically zero directions there, so they agree to round-off), then the `prec` form timed
        like the main step and checked against its own FP64 amplitudes;
    (2) a capped case where the forms differ: a 3x4 grid, 8 cycles of Haar-random two-qubit
        gates, every gate in the ket (split 8), bonds capped at chi = 4. All 4096 amplitudes of
        each form against the untruncated FP64 amplitudes (exact), as the fidelity
        |<exact|approx>|^2 / <approx|approx>.
    Returns the compact section and the two-sided FP64 amplitudes of the first 192 bitstrings."""
    import gen
    B = len(packed)
    c2 = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c2, w.split, w.chi, w.cutoff, compress="two_sided")
    # the headline plan keeps its workspace (all 65536 bitstrings in one batch) meanwhile: this
    # plan gets half the budget and runs the batch in two
    p2 = tn.tn_path(c2, layers=2, mem_budget_bytes=min(mem_gib, 48.0) * 2 ** 30)
    rms = float(np.sqrt(np.mean(np.abs(a64) ** 2)))
    d64 = tn.tn_amplitudes(p2, packed[idx], "fp64")
    bits_dev = torch.from_numpy(packed.view(np.int64).copy()).cuda()
    out = torch.empty(B, dtype=torch.complex128, device="cuda")
    ts, _, _ = form_run(tn, np, torch, c2, w, p2, bits_dev, out, prec, steps, warmup, flush)
    rel = np.abs(out.cpu().numpy()[idx] - d64) / float(np.sqrt(np.mean(np.abs(d64) ** 2)))
    ok = float(np.mean(rel <= TOL))
    d64_first = tn.tn_amplitudes(p2, packed[:192], "fp64")    # the CPU baseline's sample
    res = {"fp64_vs_one_sided_fp64": r3(float(np.max(np.abs(d64 - a64)) / rms)),
           prec: r3({"value": B / ts * ok, "ms_per_step": 1000 * ts, "max_rel_err_vs_fp64": float(rel.max())})}
    del p2, out
    g = gen.grid(3, 4)
    gates = gen.rqc(g, 8, gen.rng(43, 1), twoq="haar", oneq="haar")
    allbits = gen.all_bitstrings(12)
    amps = {}
    for label, chi, comp in (("exact", 0, "one_sided"), ("one_sided", 4, "one_sided"), ("two_sided", 4, "two_sided")):
        cc = tn.tn_build(12, g.edges, gates)
        tn.tn_evolve_two_sided(cc, 8, chi, 1e-12, compress=comp)
        amps[label] = tn.tn_amplitudes(tn.tn_path(cc), allbits, "fp64")
    ex = amps["exact"]
    fid = {}
    for label in ("one_sided", "two_sided"):
        a = amps[label]
        fid[label] = r3(float(abs(np.vdot(ex, a)) ** 2 / (np.vdot(a, a).real * np.vdot(ex, ex).real)))
    res["capped_3x4_haar_chi4_fidelity"] = fid
    return res, d64_first


def kernel_table(prof, steps):
    return {k: {"ms_per_step": v["ms"] / steps, "launches_per_step": v["launches"] / steps,
                "GB/s": v["bytes"] / max(v["ms"], 1e-9) / 1e6, "TFLOP/s": v["flops"] / max(v["ms"], 1e-9) / 1e9}
            for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x6",
                    choices=["fp64", "fp32", "tf32", "tf32x3", "bf16x3", "bf16x6", "tf32x6"])
    ap.add_argument("--bits", type=int, default=65536)
    ap.add_argument("--check-bits", type=int, default=1024, help="bitstrings re-run on the FP64 path")
    ap.add_argument("--cpu-sample", type=int, default=192, help="bitstrings timed on the CPU oracle")
    ap.add_argument("--ref-sample", type=int, default=64, help="reference arm: oracle bitstrings per step")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-only", action="store_true", help="short run for ncu captures")
    ap.add_argument("--profile-network", default="double_layer", choices=["double_layer", "overlap"],
                    help="with --profile-only: the network whose step is profiled")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="serving stream length (0: skip)")
    ap.add_argument("--serve", action="store_true", help="serving comparison only: BF16x6 vs FP64 (one line)")
    ap.add_argument("--no-tune", action="store_true", help="keep the shape heuristic's step kernels")
    ap.add_argument("--force-kernel", action="append", default=[], metavar="STEP=NAME",
                    help="with --profile-only: run plan step STEP (index of tn_plan_details) on kernel NAME")
    ap.add_argument("--mem-gib", type=float, default=96.0, help="device memory budget of the plan's batches")
    ap.add_argument("--no-batch", action="store_true", help="skip the 32-circuit batched-graph measurement")
    ap.add_argument("--no-two-sided", action="store_true", help="skip the two-sided compression section")
    ap.add_argument("--no-overlap", action="store_true",
                    help="skip the overlap-network section (per-qubit tensors of Eq. overlap, TMA-fed tcgen05 steps)")
    args = ap.parse_args()
    rank, world, local = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import gen
    assert args.warmup >= 1
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", rank=rank, world_size=world, device_id=torch.device("cuda", local))
    from paper_2011_02621_gb300 import build
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    from paper_2011_02621_gb300 import tn

    if args.serve:
        if rank == 0:
            plans, a = serving_run(tn, np, "bf16x6", max(args.serve_seconds, 1.0))
            _, b = serving_run(tn, np, "fp64", max(args.serve_seconds, 1.0), plans=plans)
            print(json.dumps({"metric": "serving p50/p99 latency and amplitudes/s, 104q d8 / 53q d10 / 20q d14 mix",
                              "unit": "s", "n_gpus": 1, "data": "synthetic", "caps": dict(SERVE_CLASSES),
                              "bf16x6": a, "fp64": b}))
        return 0

    w = gen.workload("syc53", n_bits=args.bits)
    bits_np = _rank_bits(w, rank)                 # weak scaling: each rank its own bitstrings
    B = len(bits_np)
    packed = tn.pack_bits(bits_np)
    stream = torch.cuda.current_stream()
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff)
    # the double-layer network with joined partial paths: the fastest plan of the library
    overlap_only = args.profile_only and args.profile_network == "overlap"
    plan = tn.tn_path(c, layers=1 if overlap_only else 2, mem_budget_bytes=args.mem_gib * 2 ** 30)
    info = plan.info
    tuned = None if args.no_tune else tn.tn_autotune(plan, args.prec, B, stream=stream)
    if args.force_kernel:
        if not args.profile_only:
            raise SystemExit("--force-kernel is a profiling option (with --profile-only)")
        ks = tn.tn_plan_kernels(plan, args.prec)
        for fk in args.force_kernel:
            i, name = fk.split("=", 1)
            ks[int(i)] = name
        tn.tn_plan_set_kernels(plan, args.prec, ks)
    bits_dev = torch.from_numpy(packed.view(np.int64).copy()).cuda()
    out_dev = torch.empty(B, dtype=torch.complex128, device="cuda")
    bits_pin = torch.from_numpy(packed.view(np.int64).copy()).pin_memory()
    out_pin = torch.empty(B, dtype=torch.complex128).pin_memory()
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")   # 256 MB > 129 MB L2

    def step(bits, out):
        tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff, stream)
        tn.tn_amplitudes(plan, bits, args.prec, out=out, stream=stream)

    def timed(steps, bits, out):
        total = 0.0
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(bits, out)
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1) / 1000.0
        return total

    for _ in range(args.warmup):
        step(bits_dev, out_dev)
    torch.cuda.synchronize()
    if args.profile_only:
        # one step inside a profiler range (ncu --profile-from-start off captures just this step)
        torch.cuda.profiler.start()
        step(bits_dev, out_dev)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        if rank == 0:
            ks = tn.tn_plan_kernels(plan, args.prec)
            _, _, mkn = tn.tn_plan_details(plan)
            print(json.dumps({"profile_only": True, "info": info, "bitstrings": B, "chunk": info["chunk_bitstrings"],
                              "steps": [[int(x) for x in r] for r in mkn], "kernels": ks}))
        return 0

    clocks = Clocks(local)
    clocks.start()
    tn.tn_launch_count(reset=True)
    tn.tn_profile_enable(True)
    t_dev = timed(args.steps, bits_dev, out_dev)
    prof = tn.tn_profile_read()
    tn.tn_profile_enable(False)
    launches = tn.tn_launch_count() // args.steps
    clk = clocks.stop()
    a_tc = out_dev.cpu().numpy()
    # end to end through the public call with pinned host buffers (copies inside the timed region)
    timed(1, bits_pin, out_pin)
    t_e2e = timed(args.steps, bits_pin, out_pin)
    if dist:
        t = torch.tensor([t_dev, t_e2e], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_dev, t_e2e = float(t[0]), float(t[1])

    # accuracy: amplitudes spread over the whole batch, against the plain FP64 GPU contraction of
    # the overlap network (another network and other kernels); only those within 1e-5 count
    nchk = min(args.check_bits, B)
    idx = np.unique(np.linspace(0, B - 1, nchk).astype(np.int64))
    p_ov = tn.tn_path(c, mem_budget_bytes=32.0 * 2 ** 30)
    t0 = time.perf_counter()
    a64 = tn.tn_amplitudes(p_ov, packed[idx], "fp64")
    t_ov64 = time.perf_counter() - t0
    rms = float(np.sqrt(np.mean(np.abs(a64) ** 2)))
    rel = np.abs(a_tc[idx] - a64) / rms
    ok_frac = float(np.mean(rel <= TOL))
    if dist:
        t = torch.tensor([ok_frac], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        ok_frac = float(t[0])
    value = world * B * args.steps / t_dev * ok_frac
    e2e_value = world * B * args.steps / t_e2e * ok_frac
    if rank != 0:
        return 0

    pk = peaks()
    roof = roofline(prof, args.steps, args.prec, pk, B)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "c128", "fp32": "c64"}.get(args.prec, "c64/" + args.prec),
        "data": "synthetic", "gpu_launches": launches,
        "config": {"workload": WORKLOAD, "bitstrings_per_gpu": B, "precision": args.prec,
                   "network": "double layer, joined paths", "l2": "256 MB flushed between steps",
                   "plan": r3({k: info[k] for k in ("n_steps", "n_slices", "cmacs", "bytes_c64", "max_intermediate",
                                                    "chunk_bitstrings")})},
        "contraction_tflops": r3(world * B * args.steps * info["flops"] / t_dev / 1e12),
        "accuracy": {"checked": int(len(idx)), "within_1e-5": ok_frac, "max_rel_err_vs_fp64": r3(float(rel.max())),
                     "ref": "FP64 overlap network, samples spread over the batch"},
        "roofline": {k: (r3(v) if k not in ("kernel", "peak_source", "bound", "unit") else v) for k, v in roof.items()},
        "kernels_ms_per_step": top_kernels(prof, args.steps),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(packed.nbytes),
                "d2h_bytes_per_step": int(B * 16)},
        "clocks": clk,
    }
    if tuned is not None:
        line["config"]["step_kernels"] = {k: tuned.count(k) for k in sorted(set(tuned))}
    sec_steps, sec_warm = min(args.steps, 3), min(args.warmup, 2)

    # the other forms on the headline plan: FP32 SIMT, and the plain FP64 GPU contraction
    forms = {}
    try:
        ts, _, _ = form_run(tn, np, torch, c, w, plan, bits_dev, out_dev, "fp32", sec_steps, sec_warm, flush)
        e32 = np.abs(out_dev.cpu().numpy()[idx] - a64) / rms
        forms["fp32"] = r3({"value": B / ts * float(np.mean(e32 <= TOL)), "max_rel_err": float(e32.max())})
        n64 = min(B, 4096)
        ts, _, _ = form_run(tn, np, torch, c, w, plan, bits_dev[:n64], out_dev[:n64], "fp64", sec_steps, 1, flush,
                            tune=False)
        forms["fp64"] = r3({"value": n64 / ts, "bitstrings": n64})
        forms["fp64_overlap"] = r3({"value": len(idx) / t_ov64, "bitstrings": int(len(idx))})
        tn.tn_autotune(plan, args.prec, B, stream=stream)      # the headline form's kernels again
    except Exception as e:  # noqa: BLE001  (recorded in the line, never ends the run)
        forms["error"] = f"{type(e).__name__}: {e}"[:200]
    line["forms"] = forms

    # the overlap network of Eq. overlap (per-qubit tensors formed, TMA-fed tcgen05 BF16x6 steps)
    if not args.no_overlap and world == 1:
        try:
            out2 = torch.empty(B, dtype=torch.complex128, device="cuda")
            ts, prof2, _ = form_run(tn, np, torch, c, w, p_ov, bits_dev, out2, "bf16x6", sec_steps, sec_warm, flush)
            e2 = np.abs(out2.cpu().numpy()[idx] - a64) / rms
            roof2 = roofline(prof2, sec_steps, "bf16x6", pk, B, network="overlap")
            line["overlap_network"] = {
                "value": r3(B / ts * float(np.mean(e2 <= TOL))), "ms_per_step": r3(1000 * ts),
                "max_rel_err": r3(float(e2.max())), "plan": r3({k: p_ov.info[k] for k in ("n_steps", "cmacs")}),
                "roofline": {k: r3(roof2[k]) for k in ("kernel", "bound", "achieved", "peak", "unit", "frac",
                                                         "traffic", "avg_launch_ms")}}
            del out2
        except Exception as e:  # noqa: BLE001
            line["overlap_network"] = {"error": f"{type(e).__name__}: {e}"[:200]}
    del p_ov
    torch.cuda.synchronize()
    from paper_2011_02621_gb300 import verify
    f_dev = verify.circuit_fidelity(w.gates, w.graph.n)
    line["verification"] = r3({"eq_fidelity": f_dev, "n_s_3_sigma": verify.required_bitstrings(f_dev),
                               "xeb_uniform_bits": verify.linear_xeb(a_tc, w.graph.n)})
    d64_two = None
    if not args.no_two_sided and world == 1:
        try:
            line["two_sided"], d64_two = two_sided_run(tn, np, torch, w, packed, idx, a64, args.prec, sec_steps,
                                                       sec_warm, flush, args.mem_gib, pk)
        except Exception as e:  # noqa: BLE001
            line["two_sided"] = {"error": f"{type(e).__name__}: {e}"[:200]}
    del plan
    torch.cuda.synchronize()
    if not args.no_batch and world == 1:
        try:
            line["batch"] = batch_run(tn, np, torch, args.prec, sec_steps, sec_warm, flush)
        except Exception as e:  # noqa: BLE001
            line["batch"] = {"error": f"{type(e).__name__}: {e}"[:200]}
    if args.serve_seconds > 0 and world == 1:
        try:
            plans, a = serving_run(tn, np, args.prec, args.serve_seconds)
            _, b = serving_run(tn, np, "fp64", args.serve_seconds, plans=plans)
            line["serving"] = {"caps": dict(SERVE_CLASSES), args.prec: a, "fp64": b}
            del plans
        except Exception as e:  # noqa: BLE001
            line["serving"] = {"error": f"{type(e).__name__}: {e}"[:200]}
    if not args.no_cpu and world == 1:
        cs = min(args.cpu_sample, B)
        r = cpu_oracle("syc53", args.bits, cs)
        err = np.abs(a_tc[:cs] - r["amps"]) / float(np.sqrt(np.mean(np.abs(r["amps"]) ** 2)))
        line["cpu_baseline"] = r3({"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                                   "sample": f"first {cs} bitstrings, ket outside the timing",
                                   "single_thread_value": r["single_thread_value"]})
        line["oracle_check"] = r3({"bitstrings": cs, "max_rel_err": float(err.max())})
        if d64_two is not None:
            # the device's two-sided FP64 amplitudes against the oracle's two-sided compression
            ct = min(cs, len(d64_two))
            r2 = cpu_oracle("syc53", args.bits, ct, compress="two_sided")
            err2 = np.abs(d64_two[:ct] - r2["amps"]) / float(np.sqrt(np.mean(np.abs(r2["amps"]) ** 2)))
            line["oracle_check_two_sided"] = r3({"bitstrings": ct, "max_rel_err": float(err2.max())})
    # the contract's keys first, the extra sections last (the end of the line is what a log tail keeps)
    first = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "gpu_launches", "config", "roofline", "cpu_baseline", "clocks", "e2e")
    ordered = {k: line[k] for k in first if k in line}
    ordered.update({k: v for k, v in line.items() if k not in ordered})
    print(json.dumps(ordered, separators=(",", ":")))
    return 0


if __name__ == "__main__":
    sys.exit(main())
