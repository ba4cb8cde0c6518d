"""Host logic of bench.py on the CPU: which roof binds a profiled kernel kind, the fraction it
reaches, the per-kernel table, and the traffic record that is valid only for the kernel sources
it was captured on."""
import json

import pytest

import bench

PK = dict(hbm_gbs=6686.0, bf16_tflops=1942.0, bf16_tflops_sustained=1735.0, source="measured")


def _prof(kind, launches, ms, bytes_, flops):
    return {kind: dict(launches=launches, ms=ms, bytes=bytes_, flops=flops),
            "slice_sum_fp64": dict(launches=launches, ms=ms / 100, bytes=1e6, flops=0.0)}


def test_tensor_bound_bf16x6_kernel_against_the_sustained_peak_over_six():
    # 10 launches in 2 steps, 1 ms each, 1e11 complex-equivalent flops and 1e9 bytes per launch
    r = bench.roofline(_prof("contract_step_tcgen05_tma", 10, 10.0, 1e10, 1e12), 2, "bf16x6", PK, 1024)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(1735.0 / 6)
    assert r["achieved"] == pytest.approx(1e11 / 1e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["launches_per_step"] == 5 and r["avg_launch_ms"] == pytest.approx(1.0)


def test_tf32_forms_take_the_nominal_ratio_of_the_bf16_peak():
    r = bench.roofline(_prof("contract_step_tcgen05", 4, 4.0, 4e9, 4e12), 1, "tf32x3", PK, 64)
    assert r["peak"] == pytest.approx(1735.0 * 1.1 / 2.25 / 3)


def test_thin_fp32_steps_are_hbm_bound():
    # intensity 2 flop/byte, below the FP32 ridge (80.5 TFLOP/s over 6.686 TB/s, about 12)
    r = bench.roofline(_prof("contract_step_fp32", 100, 50.0, 3e11, 6e11), 2, "fp32", PK, 65536)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6686.0
    assert r["achieved"] == pytest.approx(3e9 / 5e-4 / 1e9)
    assert r["traffic"] is None                    # no capture of this kernel


def test_fp64_steps_above_the_fp64_ridge_are_alu_bound():
    r = bench.roofline(_prof("contract_step_fp64", 1, 10.0, 1e8, 1e10), 1, "fp64", PK, 16)
    assert r["bound"] == "alu" and r["peak"] == 1.25


def test_kernel_table_is_sorted_by_time_per_step():
    t = bench.kernel_table({"a": dict(launches=2, ms=1.0, bytes=1e9, flops=0.0),
                            "b": dict(launches=4, ms=3.0, bytes=3e9, flops=6e12)}, 2)
    assert list(t) == ["b", "a"]
    assert t["b"]["ms_per_step"] == 1.5 and t["b"]["launches_per_step"] == 2
    assert t["b"]["GB/s"] == pytest.approx(1000.0) and t["b"]["TFLOP/s"] == pytest.approx(2000.0)


def test_traffic_record_is_dropped_when_the_kernel_sources_change(tmp_path, monkeypatch):
    """A network's record gives the kernel's DRAM bytes per algorithmic byte; the roofline scales it to
    the run's algorithmic bytes per launch, and drops it once the kernel's sources hash differently."""
    kind = "contract_step_tcgen05_tma"
    rec = {"overlap": {kind: {"dram_over_algorithmic": 0.9, "source_sha": bench.source_sha(kind)}}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_sha", lambda kind=None: rec["overlap"][kind]["source_sha"])
    assert bench.traffic_record(kind, "overlap")["dram_over_algorithmic"] == 0.9
    assert bench.traffic_record(kind, "double_layer") is None           # another network's plan
    r = bench.roofline(_prof(kind, 10, 10.0, 1e10, 1e12), 2, "bf16x6", bench.peaks(), 1000, network="overlap")
    assert r["traffic"] == pytest.approx(0.9 * 1e10 / 10)               # per launch
    monkeypatch.setattr(bench, "source_sha", lambda kind=None: "0" * 16)
    assert bench.traffic_record(kind, "overlap") is None
