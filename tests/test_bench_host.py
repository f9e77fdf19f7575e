"""Host-side bookkeeping of bench.py, checked on CPU against hand counts:
clock-record parsing, the per-kernel units of a W-cycle, algorithmic bytes,
the roofline object and the derived FP64 peaks."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _levels(octs, cache):
    lo = [0] * 16
    lc = [0] * 16
    for l, n in octs.items():
        lo[l] = n
    for l, n in cache.items():
        lc[l] = n
    return {"level_octs": lo, "level_cache": lc}


def test_clock_summary_parses_reasons_and_medians():
    s = bench.ClockSampler(0)
    s.lines = [
        "0, 2070, 2070, 600.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 650.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, 1500, 2070, 700.0, 0x8, Active, Not Active, Not Active, Not Active",
    ]
    out = s.summary()
    assert out["samples"] == 4
    assert out["sm_mhz"] == pytest.approx((1980 + 2070) / 2)
    assert out["sm_max_mhz"] == 2070
    assert out["power_w_max"] == 900.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    empty = bench.ClockSampler(0)
    assert empty.summary()["samples"] == 0


def test_kernel_units_count_the_w_cycle():
    # levels 3 (base, 8 octs), 4 (5 octs, 3 ghost octs), 5 (2 octs, 4 ghosts)
    info = _levels({3: 8, 4: 5, 5: 2}, {4: 3, 5: 4})
    loc, real, ghost, fine = bench.kernel_units(info, 3)
    # level l runs 2^(l-3) times per coarse step
    assert real == 8 * (8 * 1 + 5 * 2 + 2 * 4)
    assert loc == 8 * ((8 + 0) * 1 + (5 + 3) * 2 + (2 + 4) * 4)
    assert ghost == 3 * 2 + 4 * 4
    assert fine == 5 * 2 + 2 * 4


def test_kernel_traffic_words_per_unit():
    info = _levels({3: 8, 4: 5}, {4: 3})
    loc, real, ghost, fine = bench.kernel_units(info, 3)
    w = 8
    t = bench.kernel_traffic(info, 3, w, fused=False)
    assert t == {"prolong": ghost * 75 * w, "reflux_restrict": ghost * 130 * w + fine * 45 * w,
                 "prim": loc * 10 * w, "predict": loc * 25 * w, "flux": loc * 35 * w,
                 "update": real * (25 * w + 4)}
    t4 = bench.kernel_traffic(info, 3, 4, fused=True)
    assert set(t4) == {"prolong", "reflux_restrict", "predict", "flux"}
    assert t4["flux"] == loc * 20 * 4 + real * (10 * 4 + 4)


def test_roofline_of_the_dominant_kernel():
    info = _levels({3: 8, 4: 5}, {4: 3})
    loc, real, _, _ = bench.kernel_units(info, 3)
    steps = 10
    # flux dominates: 20 launches (2 per step) taking 4 ms in all
    res = {"info": info, "steps": steps,
           "kernels": {"flux": (4.0, 20), "predict": (1.0, 20), "update": (0.5, 20)}}
    traffic = bench.kernel_traffic(info, 3, 4, fused=True)
    rl, table = bench.roofline(res, 4, 3, 6000.0, "measured")
    assert list(table) == ["flux", "predict", "update"]
    assert table["flux"]["share"] == pytest.approx(4.0 / 5.5, abs=1e-4)
    bytes_per_launch = traffic["flux"] * steps / 20
    avg_s = 4.0 / 20 * 1e-3
    assert rl["kernel"] == "flux" and rl["bound"] == "hbm"
    assert rl["algorithmic_bytes_per_launch"] == int(bytes_per_launch)
    assert rl["achieved"] == pytest.approx(bytes_per_launch / avg_s / 1e9, abs=0.05)
    assert rl["frac"] == pytest.approx(rl["achieved"] / 6000.0, abs=1e-4)
    assert rl["traffic"] == int(bench.FLUX_DRAM_BYTES_PER_CELL[4] * real * steps / 20)
    # FP64: the flux kernel against the FP64 pipe, flops per real cell
    peak = bench.fp64_peak_derived(2070.0)
    rl8, _ = bench.roofline(res, 8, 3, 6000.0, "measured", fp64_tflops=peak, dgemm=1.1, sm_mhz=2070.0)
    flops = bench.FLUX_FP64_FLOPS_PER_CELL * real * steps / 20
    assert rl8["bound"] == "alu" and rl8["unit"] == "TFLOP/s"
    assert rl8["achieved"] == pytest.approx(flops / avg_s / 1e12, abs=1e-4)
    assert rl8["frac"] == pytest.approx(rl8["achieved"] / peak, abs=1e-4)
    assert rl8["hbm_view"]["bound"] == "hbm"


def test_derived_peaks():
    # 152 SMs x 2 FP64 FMA x 2 flops x 2.07 GHz
    assert bench.fp64_peak_derived(2070.0) == pytest.approx(1.25856, abs=1e-5)
    cic = {"fp64": {"cic_atomic_roofline": {"achieved": 500.0}}}
    bench.cic_alu_peak(cic, 2070.0)
    rl = cic["fp64"]["cic_atomic_roofline"]
    assert rl["peak"] == pytest.approx(152 * 2 * 2.07e9 / 1e9, abs=0.05)
    assert rl["frac"] == pytest.approx(500.0 / rl["peak"], abs=1e-4)


def test_measured_peaks_are_read():
    gbs, src = bench.load_peaks()
    assert src in ("measured", "fallback")
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert src == "measured" and gbs > 1000.0


def test_all_core_oracle_baseline_runs_replicas():
    """One oracle replica per host core, one coarse step each: a positive
    rate over all cores, and a dictionary (never a hang) on any failure."""
    out = bench.cpu_baseline_all_cores(3692312, 1)
    assert "unavailable" not in out, out
    assert out["cores"] == (os.cpu_count() or 1) and out["kind"] == "oracle"
    assert out["value"] > 0
