"""Host-side helpers of bench.py (no GPU): the FP64 ALU peak, the parse of
the committed ncu summary, the per-level split of the barrier stamps and the
parse of the sampled clocks with their throttle reasons."""
import json
import os
import tempfile

import pytest

import bench


def test_fp64_alu_peak_from_unit_counts():
    # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
    assert bench.fp64_peak(152, 2070) == pytest.approx(1.259e12, rel=1e-3)


def test_profiled_traffic_follows_the_committed_capture():
    rec = json.load(open(bench.TRAFFIC))
    got = bench.profiled_traffic(16384)
    if rec["kernel_sources_sha256"] == bench.csrc_digest():
        assert got == pytest.approx(rec["dram_bytes_per_block"] * 16384)
    else:  # the kernels changed since the capture: no traffic figure
        assert got is None


def test_kernel_rooflines_from_class_times():
    # residual: 6 n^2 d N flops per launch; two launches of 1 ms each
    # over 2 steps: 4 residual launches (2 per step) of 1 ms, 2 corrections
    kt = {"residual": (4.0, 4), "correction": (4.0, 2), "solve": (0.0, 0), "factor": (30.0, 74)}
    units = {"residual": 2, "correction": 1, "factor": 1}
    r = bench.kernel_rooflines(kt, 2, units, N=100, n=8, d=2, mode="fp32_ir", sms=152, mhz=2070)
    assert set(r) == {"residual", "correction", "factor"}
    assert r["residual"]["achieved"] == pytest.approx(6 * 64 * 2 * 100 / 1e-3 / 1e12)
    # a factorisation split over many launches still counts once per step
    assert r["factor"]["ms_per_unit"] == pytest.approx(15.0)
    assert r["residual"]["frac"] == pytest.approx(r["residual"]["achieved"] / r["residual"]["peak"])
    assert r["correction"]["bound"] == "hbm" and r["correction"]["unit"] == "GB/s"


def test_phase_split_maps_stamps_to_levels():
    L = 2
    # start, A0, B0, A1, B1, top, C1 (ns)
    stamps = [0, 1000, 3000, 6000, 10000, 15000, 21000]
    out = bench.phase_split(stamps, L, launch_ms=0.030)
    assert out["A"] == [1.0, 3.0] and out["B"] == [2.0, 4.0]
    assert out["top"] == 5.0 and out["C"] == [6.0]
    assert out["edges"] == pytest.approx(30.0 - 21.0)
    assert bench.phase_split(stamps[:4], L, 0.01) is None


def test_clock_summary_reports_throttle_reasons():
    cs = bench.ClockSampler(0)
    cs.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    rows = [
        "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1390.2, 0x8, Active, Not Active, Not Active, Active",
        "garbage line",
    ]
    cs.f.write("\n".join(rows) + "\n")
    cs.f.flush()
    s = cs.summary()
    assert not os.path.exists(cs.f.name)
    assert s["samples"] == 3 and s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert s["power_w_max"] == pytest.approx(1390.2)
