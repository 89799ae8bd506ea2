"""Host logic of the benchmark (no device): the roofline arithmetic, the
clock-record parsing that decides whether a run is kept, and the reference
arm's JSON line (the FP64 oracle on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_sfu_roofline_counts_results_per_clock():
    """64 normals (Box-Muller: lg2, sqrt, sin, cos per pair = 2 slow results
    each) and 64 ex2 per path-step: 128 / 16 + 64 / 32 = 10 SM-cycles, so the
    peak is SMs x clock / 10 path-steps/s."""
    hw = bench.Hw(152)
    hw.hz = 2.0e9
    r = hw.sfu(1.5e10, normals=64, ex2=64)
    assert r["peak"] == pytest.approx(152 * 2.0e9 / 10.0)
    assert r["frac"] == pytest.approx(1.5e10 / r["peak"])
    assert r["bound"] == "alu" and r["unit"] == bench.UNIT


def test_tensor_and_fma_rooflines():
    hw = bench.Hw(152)
    hw.hz, hw.bf16 = 2.0e9, 2.0e15
    for dtype, ratio in (("bf16", 1.0), ("fp16", 1.0), ("fp8", 2.0), ("tf32", 0.5)):
        t = hw.tensor(5.0e14, dtype)
        assert t["peak"] == pytest.approx(2000.0 * ratio) and t["frac"] == pytest.approx(0.25 / ratio)
    f = hw.fma(1.0e13)
    assert f["peak"] == pytest.approx(152 * 128 * 2.0e9 / 1e12)
    assert f["frac"] == pytest.approx(1.0e13 / (152 * 128 * 2.0e9))


def test_clock_summary_reads_reasons_and_median():
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2040, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line",
               "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = c.summary()
    assert s["sm_mhz"] == 2040.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = ["0, 1500, 2070, 700, 0x48, Active, Not Active, Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.lines = []
    assert c.summary()["sm_mhz"] is None


def test_peaks_come_from_the_measured_file():
    pk, kind = bench.peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured"
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            assert pk == json.load(f)
    else:
        assert kind == "fallback" and pk["hbm_gbs"] == 6800.0 and pk["bf16_tflops"] == 1900.0


@pytest.mark.slow
def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference: one JSON line, the oracle timed on the host
    cores over a bounded prefix of the headline workload, with the keys the
    base contract and its reference arm ask for."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["dtype"] == "f64" and line["steps"] == 1
    assert line["warmup"] == 3 and line["value"] > 0 and line["config"]["workload"] == bench.WORKLOAD
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert 256 <= line["config"]["paths_sampled"] <= 1 << 16
