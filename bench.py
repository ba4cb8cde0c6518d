#!/usr/bin/env python
"""Benchmark of the TNS amplitude path on one GB300 per rank.

Workload (one "step"): the 53-qubit staggered diagonal-coupled grid (6 rows x
9 columns minus one seeded site), 10 cycles ABCDCDABAB, two-sided evolution
split after cycle 5, bonds truncated to chi = 64 or singular values below
1e-8 s_0; one step = the ket evolution + the batched bra evolution, overlap
network, sliced contraction and FP64 slice sum for 65536 seeded random
bitstrings. Synthetic seeded inputs stand in for the Sycamore layout and
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
def traffic_record(kind):
    """DRAM bytes of `kind` per bitstring and step, from a committed ncu capture of a small case
    (profiles/traffic.json), if the kernel sources are unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    rec = d.get(kind)
    if not rec or rec.get("source_sha") != source_sha():
        return None
    return rec


TRAFFIC_SOURCES = ("tc_tma.cu", "tn_device.h", "tn_internal.h")   # the TMA step kernel and its headers


def source_sha():
    """Hash of the TMA step kernel's sources: a traffic record taken on other sources is stale."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2011_02621_gb300", "csrc")
    for f in TRAFFIC_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------
# serving: a seeded Poisson request stream over three circuit classes
# ---------------------------------------------------------------------------
SERVE_CLASSES = (("syc104", 4096), ("syc53", 65536), ("grid20", 16))   # (workload, size cap)


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
    res = {"workload": f"32 circuits on seeded random 3-regular graphs, 24-40 qubits, {depth} cycles "
                       "(Haar SU(2) + fSim(pi/2, pi/6) per edge colour), 1024 bitstrings each, "
                       + ("largest chi with no cut at 2^24" if truncated else "untruncated"),
           "precision": prec, "amplitudes": total, "value": total / t_graph * scale, "unit": UNIT,
           "ms_per_launch": 1000 * t_graph, "graph_kernels": info["graph_kernels"],
           "device_bytes": info["device_bytes"],
           "vs_fp64": {"amplitudes_compared": checked, "within_1e-5": frac, "max_rel_err": worst},
           "chi_per_circuit": chis if truncated else None, "contraction_tflops": 8 * cmacs / t_graph / 1e12,
           "sequential_calls": {"value": total / t_seq * scale, "ms": 1000 * t_seq},
           "e2e": {"value": total / t_e2e * scale, "unit": UNIT, "h2d_bytes_per_step": int(flat.nbytes),
                   "d2h_bytes_per_step": int(total * 16)}}
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
            opts = {"max_intermediate": 1 << 22} if name == "grid20" else {}
            plans[name] = (tn.tn_path(c, mem_budget_bytes=4.0 * 2 ** 30, **opts), w.graph.n, cap)
    # capacity (amplitudes/s) per class in this form, from one batch each
    capacity = {}
    for name, (p, nq, cap) in plans.items():
        nb = max(4, min(cap, 1024 if name != "grid20" else 8))
        bits = gen.bitstrings(nq, nb, gen.rng(seed, 9))
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
    return plans, {"precision": prec, "requests": len(tickets), "offered_load": load,
                   "arrival_rate_per_s": lam, "seconds": seconds,
                   "amplitudes": st["amplitudes"], "amplitudes_per_s": st["amplitudes"] / wall,
                   "p50_latency_s": st["p50_latency_s"], "p99_latency_s": st["p99_latency_s"],
                   "max_inflight_seen": st["max_inflight_seen"],
                   "capacity_amplitudes_per_s": {k: round(v, 1) for k, v in capacity.items()},
                   "size_caps": dict(SERVE_CLASSES)}


def roofline(prof, steps, prec, pk, n_bits):
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
    tr = traffic_record(kind)
    # scaled to this run's launches by the bitstrings they process (traffic grows in proportion)
    roof["traffic"] = tr["dram_bytes_per_bitstring_step"] * n_bits / (rec["launches"] / steps) if tr else None
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


def double_layer_run(tn, np, torch, c, w, packed, a64, steps, warmup, flush, mem_gib, pk):
    """The same amplitudes from the double-layer network: every qubit's ket and bra tensors stay
    two nodes joined by the physical index, and the path Algorithm 1 finds on that network absorbs
    them one at a time, instead of first forming the per-qubit overlap tensors of Eq. overlap.
    FP64 on the first len(a64) bitstrings against the overlap network's FP64 amplitudes a64 (equal
    up to round-off), then the FP32 form (its steps are thin and memory-bound, so no tensor-core
    form) with autotuned SIMT step kernels, timed like the main step (ket evolution + amplitudes,
    L2 flushed between steps) and checked against a64."""
    stream = torch.cuda.current_stream()
    B = len(packed)
    nchk = len(a64)
    t0 = time.perf_counter()
    p2 = tn.tn_path(c, layers=2, mem_budget_bytes=mem_gib * 2 ** 30)
    info = p2.info
    res = {"network": "double layer: ket and bra tensors as separate nodes joined by the physical index",
           "plan_seconds": time.perf_counter() - t0,
           "plan": {k: info[k] for k in ("n_steps", "n_cuts", "n_slices", "cmacs", "flops", "bytes_c64",
                                         "max_intermediate", "chunk_bitstrings")}}
    rms = float(np.sqrt(np.mean(np.abs(a64) ** 2)))
    d64 = tn.tn_amplitudes(p2, packed[:nchk], "fp64")
    res["fp64_vs_overlap_fp64"] = {"checked": nchk, "max_rel_err": float(np.max(np.abs(d64 - a64)) / rms)}
    tuned = tn.tn_autotune(p2, "fp32", B, stream=stream)
    bits_dev = torch.from_numpy(packed.view(np.int64).copy()).cuda()
    out = torch.empty(B, dtype=torch.complex128, device="cuda")

    def step():
        tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff, stream)
        tn.tn_amplitudes(p2, bits_dev, "fp32", out=out, stream=stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    tn.tn_launch_count(reset=True)
    tn.tn_profile_enable(True)
    total = timed_section(torch, stream, step, steps, 0, flush)
    prof = tn.tn_profile_read()
    tn.tn_profile_enable(False)
    launches = tn.tn_launch_count() // steps
    a32 = out[:nchk].cpu().numpy()
    rel = np.abs(a32 - a64) / rms
    ok = float(np.mean(rel <= TOL))
    res["fp32"] = {"value": B * steps / total * ok, "unit": UNIT, "ms_per_step": 1000 * total / steps,
                   "bitstrings_per_step": B, "gpu_launches": launches,
                   "contraction_tflops": B * steps * info["flops"] / total / 1e12,
                   "accuracy": {"checked": nchk, "within_1e-5": ok, "max_rel_err_vs_fp64": float(rel.max())},
                   "roofline": roofline(prof, steps, "fp32", pk, B), "kernels": kernel_table(prof, steps),
                   "step_kernels": {k: tuned.count(k) for k in sorted(set(tuned))}}
    return res


def two_sided_run(tn, np, torch, w, packed, a64, prec, steps, warmup, flush, mem_gib, pk):
    """The two-sided bond compression (the singular values of the local product of a gate's two
    endpoints, a variant of Eqs. svd/svd2 the paper does not use) on the device:
    (1) the same workload with both halves compressed two-sided: FP64 on the first len(a64)
        bitstrings against the one-sided FP64 amplitudes a64, then the `prec` form timed like the
        main step and checked against its own FP64 amplitudes;
    (2) a capped case where the forms differ: a 3x4 grid, 8 cycles of Haar-random two-qubit
        gates, every gate in the ket (split 8), bonds capped at chi = 4. All 4096 amplitudes of
        each form against the untruncated FP64 amplitudes (exact), as the fidelity
        |<exact|approx>|^2 / <approx|approx> and the largest error relative to rms |exact|.
    Returns the section and the two-sided FP64 amplitudes of (1)."""
    import gen
    stream = torch.cuda.current_stream()
    B = len(packed)
    nchk = len(a64)
    c2 = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c2, w.split, w.chi, w.cutoff, stream, compress="two_sided")
    p2 = tn.tn_path(c2, mem_budget_bytes=mem_gib * 2 ** 30)
    rms = float(np.sqrt(np.mean(np.abs(a64) ** 2)))
    d64 = tn.tn_amplitudes(p2, packed[:nchk], "fp64")
    res = {"compression": "two-sided: two gate-kernel entries per gate (the other endpoint decomposed "
                          "whole, then the kept endpoint under the keep rule)",
           "plan": {k: p2.info[k] for k in ("n_steps", "cmacs", "max_intermediate", "chunk_bitstrings")},
           "fp64_vs_one_sided_fp64": {"checked": nchk, "max_rel_err": float(np.max(np.abs(d64 - a64)) / rms)}}
    tuned = tn.tn_autotune(p2, prec, B, stream=stream)
    bits_dev = torch.from_numpy(packed.view(np.int64).copy()).cuda()
    out = torch.empty(B, dtype=torch.complex128, device="cuda")

    def step():
        tn.tn_evolve_two_sided(c2, w.split, w.chi, w.cutoff, stream)
        tn.tn_amplitudes(p2, bits_dev, prec, out=out, stream=stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    tn.tn_profile_enable(True)
    total = timed_section(torch, stream, step, steps, 0, flush)
    prof = tn.tn_profile_read()
    tn.tn_profile_enable(False)
    rel = np.abs(out[:nchk].cpu().numpy() - d64) / float(np.sqrt(np.mean(np.abs(d64) ** 2)))
    ok = float(np.mean(rel <= TOL))
    res[prec] = {"value": B * steps / total * ok, "unit": UNIT, "ms_per_step": 1000 * total / steps,
                 "accuracy": {"checked": nchk, "within_1e-5": ok, "max_rel_err_vs_fp64": float(rel.max())},
                 "kernels": kernel_table(prof, steps),
                 "step_kernels": {k: tuned.count(k) for k in sorted(set(tuned))}}
    del p2
    # (2) a capped case: exact amplitudes from the untruncated FP64 path on the same device
    g = gen.grid(3, 4)
    gates = gen.rqc(g, 8, gen.rng(43, 1), twoq="haar", oneq="haar")
    allbits = gen.all_bitstrings(12)
    amps = {}
    for label, chi, comp in (("exact", 0, "one_sided"), ("one_sided", 4, "one_sided"), ("two_sided", 4, "two_sided")):
        cc = tn.tn_build(12, g.edges, gates)
        tn.tn_evolve_two_sided(cc, 8, chi, 1e-12, stream, compress=comp)
        amps[label] = tn.tn_amplitudes(tn.tn_path(cc), allbits, "fp64")
    ex = amps["exact"]
    capped = {"workload": "3x4 grid, 8 cycles of Haar-random two-qubit gates and Haar SU(2), split 8, chi 4, "
                          "all 4096 bitstrings", "norm_exact": float(np.sum(np.abs(ex) ** 2))}
    for label in ("one_sided", "two_sided"):
        a = amps[label]
        capped[label] = {"fidelity": float(abs(np.vdot(ex, a)) ** 2 / (np.vdot(a, a).real * np.vdot(ex, ex).real)),
                         "max_rel_err_vs_exact": float(np.max(np.abs(a - ex)) / np.sqrt(np.mean(np.abs(ex) ** 2)))}
    res["capped_3x4_haar_chi4"] = capped
    return res, d64


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
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="serving stream length (0: skip)")
    ap.add_argument("--serve", action="store_true", help="serving comparison only: BF16x6 vs FP64 (one line)")
    ap.add_argument("--no-tune", action="store_true", help="keep the shape heuristic's step kernels")
    ap.add_argument("--mem-gib", type=float, default=32.0, help="device memory budget of the plan's batches")
    ap.add_argument("--no-batch", action="store_true", help="skip the 32-circuit batched-graph measurement")
    ap.add_argument("--no-two-sided", action="store_true", help="skip the two-sided compression section")
    ap.add_argument("--no-double-layer", action="store_true",
                    help="skip the double-layer network section (ket and bra tensors as separate nodes)")
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
                              "unit": "s", "n_gpus": 1, "data": "synthetic", "tensor_core": a, "fp64": b}))
        return 0

    w = gen.workload("syc53", n_bits=args.bits)
    bits_np = _rank_bits(w, rank)                 # weak scaling: each rank its own bitstrings
    B = len(bits_np)
    packed = tn.pack_bits(bits_np)
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates)
    tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff)
    plan = tn.tn_path(c, mem_budget_bytes=args.mem_gib * 2 ** 30)
    info = plan.info
    stream = torch.cuda.current_stream()
    tuned = None if args.no_tune else tn.tn_autotune(plan, args.prec, B, stream=stream)
    bits_dev = torch.from_numpy(packed.view(np.int64).copy()).cuda()
    out_dev = torch.empty(B, dtype=torch.complex128, device="cuda")
    bits_pin = torch.from_numpy(packed.view(np.int64).copy()).pin_memory()
    out_pin = torch.empty(B, dtype=torch.complex128).pin_memory()
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")   # 256 MB > 129 MB L2

    def step(bits, out):
        tn.tn_evolve_two_sided(c, w.split, w.chi, w.cutoff, stream)
        tn.tn_amplitudes(plan, bits, args.prec, out=out, stream=stream)

    def timed(steps, bits, out, profile=False):
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
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        step(bits_dev, out_dev)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        if rank == 0:
            print(json.dumps({"profile_only": True, "info": info}))
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

    # accuracy: re-run a sample on the FP64 path; only amplitudes within 1e-5 of FP64 count
    nchk = min(args.check_bits, B)
    a64 = tn.tn_amplitudes(plan, packed[:nchk], "fp64")
    rms = float(np.sqrt(np.mean(np.abs(a64) ** 2)))
    rel = np.abs(a_tc[:nchk] - a64) / rms
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
    kernels = kernel_table(prof, args.steps)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "c128", "fp32": "c64"}.get(args.prec, "c64/" + args.prec),
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "bitstrings_per_gpu": B, "precision": args.prec,
                   "l2": "256 MB buffer written between timed steps; intermediates exceed L2",
                   "plan": {k: info[k] for k in ("n_steps", "n_cuts", "n_slices", "cmacs", "flops", "bytes_c64",
                                                 "max_intermediate", "chunk_bitstrings", "max_rank_used")}},
        "contraction_tflops": world * B * args.steps * info["flops"] / t_dev / 1e12,
        "accuracy": {"checked": nchk, "within_1e-5": ok_frac, "max_rel_err_vs_fp64": float(rel.max())},
        "roofline": roof,
        "kernels": kernels,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(packed.nbytes),
                "d2h_bytes_per_step": int(B * 16)},
        "clocks": clk,
    }
    if tuned is not None:
        line["config"]["step_kernels"] = {k: tuned.count(k) for k in sorted(set(tuned))}
    from paper_2011_02621_gb300 import verify
    f_dev = verify.circuit_fidelity(w.gates, w.graph.n)
    line["verification"] = {"eq_fidelity_sycamore_error_rates": f_dev,
                            "required_bitstrings_3_sigma": verify.required_bitstrings(f_dev),
                            "linear_xeb_of_uniform_bitstrings": verify.linear_xeb(a_tc, w.graph.n)}
    if not args.no_batch and world == 1:
        del plan                       # its workspace goes back to the allocator first
        torch.cuda.synchronize()
        try:
            line["batch"] = batch_run(tn, np, torch, args.prec, args.steps, args.warmup, flush)
        except tn.TNError as e:
            line["batch"] = {"error": str(e)}
    if args.serve_seconds > 0 and world == 1:
        try:
            _, sv = serving_run(tn, np, args.prec, args.serve_seconds)
            line["serving"] = sv
        except tn.TNError as e:
            line["serving"] = {"error": str(e)}
    if not args.no_double_layer and world == 1:
        # last of the GPU sections: a failure here is recorded and leaves the numbers above as they are
        try:
            line["double_layer"] = double_layer_run(tn, np, torch, c, w, packed, a64, args.steps, args.warmup,
                                                    flush, args.mem_gib, pk)
        except Exception as e:  # noqa: BLE001  (recorded in the line, never ends the run)
            line["double_layer"] = {"error": f"{type(e).__name__}: {e}"}
    d64_two = None
    if not args.no_two_sided and world == 1:
        try:
            line["two_sided"], d64_two = two_sided_run(tn, np, torch, w, packed, a64, args.prec, args.steps,
                                                       args.warmup, flush, args.mem_gib, pk)
        except Exception as e:  # noqa: BLE001  (recorded in the line, never ends the run)
            line["two_sided"] = {"error": f"{type(e).__name__}: {e}"}
    if not args.no_cpu and world == 1:
        cs = min(args.cpu_sample, B)
        r = cpu_oracle("syc53", args.bits, cs)
        err = np.abs(a_tc[:cs] - r["amps"]) / float(np.sqrt(np.mean(np.abs(r["amps"]) ** 2)))
        line["cpu_baseline"] = {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                                "sample": f"first {cs} of the 65536 bitstrings (ket evolution outside the timing)",
                                "single_thread_value": r["single_thread_value"], "wall_s": r["wall_s"]}
        line["oracle_check"] = {"bitstrings": cs, "max_rel_err": float(err.max())}
        if d64_two is not None:
            # the device's two-sided FP64 amplitudes against the oracle's two-sided compression
            ct = min(cs, len(d64_two))
            r2 = cpu_oracle("syc53", args.bits, ct, compress="two_sided")
            err2 = np.abs(d64_two[:ct] - r2["amps"]) / float(np.sqrt(np.mean(np.abs(r2["amps"]) ** 2)))
            line["oracle_check_two_sided"] = {"bitstrings": ct, "precision": "fp64", "max_rel_err": float(err2.max()),
                                              "oracle_value": r2["value"]}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
