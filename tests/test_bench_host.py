"""Host logic of bench.py (no GPU): the roofline objects built from traced
kernel times and work counts, and the clock summary that qualifies a run."""
import json
import os

import pytest

import bench

PK = {"hbm_gbs": 6790.0, "bf16_tflops": 1864.9, "bf16_tflops_sustained": 1702.8}


def _k(name, ms, launches, work, kind):
    return {"name": name, "ms": ms, "launches": launches, "work": work, "kind": kind}


def test_roofline_entry_per_kind():
    # 1 GB per launch in 1 ms: 1000 GB/s against the measured copy bandwidth
    e = bench.roofline_entry(_k("stream", 10.0, 10, 10e9, "hbm_bytes"), PK, "measured")
    assert e["bound"] == "hbm" and e["unit"] == "GB/s"
    assert e["achieved"] == pytest.approx(1000.0) and e["frac"] == pytest.approx(1000.0 / 6790.0)
    # 1.2 GFLOP per launch in 10 ms: 0.12 TFLOP/s against 152 SMs x 2 DFMA x 2 flops x 2.07 GHz
    e = bench.roofline_entry(_k("fp64", 20.0, 2, 2.4e9, "fp64_flops"), PK, "measured")
    assert e["bound"] == "alu" and e["unit"] == "TFLOP/s"
    assert e["peak"] == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)
    assert e["achieved"] == pytest.approx(0.12)
    # tensor-core work inside a long step takes the sustained figure when present
    e = bench.roofline_entry(_k("mma", 1.0, 1, 1e12, "bf16_tensor_flops"), PK, "measured")
    assert e["bound"] == "tensor" and e["peak"] == 1702.8 and e["achieved"] == pytest.approx(1000.0)
    burst = {k: v for k, v in PK.items() if k != "bf16_tflops_sustained"}
    assert bench.roofline_entry(_k("mma", 1.0, 1, 1e12, "bf16_tensor_flops"), burst, "fallback")["peak"] == 1864.9


def test_roofline_of_picks_the_dominant_kernel_and_its_traffic():
    name = "grad_eri3_kernel (fused d(mu nu|P) . Y)"
    stats = [
        _k("SCF iteration graph: tensor-core RI-K, 6 digits", 50.0, 10, 0.0, "fp64_flops"),   # not a kernel row
        _k(name, 40.0, 10, 1.9e10, "fp64_flops"),
        _k("eigh F' (refine only)", 30.0, 96, 0.0, "fp64_flops"),
        _k("fit trsm", 10.0, 10, 2.6e11, "fp64_flops"),
    ]
    r = bench.roofline_of(stats, PK, "measured")
    assert r["kernel"] == name and r["dominant_kernel"] == name
    assert r["dominant_share"] == pytest.approx(40.0 / 130.0)
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        assert r["traffic"] == json.load(f)[name]
    assert [k["kernel"] for k in r["all_kernels"]] == [name, "fit trsm"]
    # a dominant kernel without a work count: the longest one with a count is the roofline kernel
    stats[2]["ms"] = 45.0
    r = bench.roofline_of(stats, PK, "measured")
    assert r["dominant_kernel"] == "eigh F' (refine only)" and r["kernel"] == name


def test_clock_summary():
    s = bench.ClockSampler(0)
    assert s.summary()["reasons"] == ["unavailable"]
    s.rows = [["2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["1980", "2070", "1300.5", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
              ["2070", "2070", "1250.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    s.rows.append(["1500", "2070", "1400", "0x8", "Not Active", "Active", "Not Active", "Not Active"])
    assert s.summary()["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
