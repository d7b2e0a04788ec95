"""Host-side bookkeeping of bench.py that needs no GPU: the roofline fraction
and its binding unit, the error statistics against the oracle, the masked
loss of the finite-difference check, the whole-job rate, and the clock
sampler (against a stand-in for nvidia-smi's query loop)."""
import math
import sys
import time

import numpy as np
import pytest

import bench

CEIL = {"gather_walk_TBs": 40.0, "gather_tile_TBs": 30.0, "gather_random_TBs": 4.0, "fma_f32_TFLOPs": 80.0,
        "fma_f64_TFLOPs": 1.0, "sms": 152}


def test_roofline_takes_the_larger_fraction():
    trials = 1.0e7
    # 1 ms: gather 12.8 TB/s (0.32 of 40), flops 9.8 TFLOP/s (0.1225 of 80)
    r = bench.roofline(trials, 1.0, 50.0, CEIL, "test")
    assert r["bound"] == "gather" and r["unit"] == "TB/s"
    assert math.isclose(r["achieved"], trials * bench.GATHER_BYTES_PER_TRIAL / 1e-3 / 1e12)
    assert math.isclose(r["frac"], r["achieved"] / 40.0)
    assert math.isclose(r["alu"]["frac"], trials * bench.FLOPS_PER_TRIAL / 1e-3 / 1e12 / 80.0)
    assert r["frac"] == max(r["gather"]["frac"], r["alu"]["frac"])
    assert math.isclose(r["fp64_tracer"]["achieved_TFLOPs"], trials * bench.FLOPS_PER_TRIAL_F64 / 50e-3 / 1e12)
    # an FMA ceiling low enough makes the ALU the binding unit
    r2 = bench.roofline(trials, 1.0, 50.0, dict(CEIL, fma_f32_TFLOPs=10.0), "test")
    assert r2["bound"] == "alu" and r2["unit"] == "TFLOP/s" and r2["frac"] == r2["alu"]["frac"]


def test_roofline_without_probes_uses_the_nominal_issue_rate():
    r = bench.roofline(1.0e7, 1.0, 50.0, None, "test")
    assert r["bound"] == "alu" and "probes skipped" in r["peak_source"]
    assert math.isclose(r["peak"], bench.NUM_SMS * bench.FP32_LANES_PER_SM * 2 * 2070.0e6 / 1e12, rel_tol=0.2)


def test_err_stats():
    n = 10
    ref = dict(Q=np.linspace(2.0, 11.0, n), Tw=np.linspace(-1.0, 1.0, n), face1=np.zeros(n), face2=np.ones(n),
               status=np.zeros(n))
    g = {k: np.copy(v) for k, v in ref.items()}
    g["Q"] = ref["Q"] * (1 + 1e-3)
    g["Q"][0] = np.nan  # a NaN on the GPU side is left out of the quantiles
    g["face2"][3] = 0
    sample = np.arange(n)
    e = bench.err_stats(g, ref, sample)
    assert math.isclose(e["q_rel_median"], 1e-3, rel_tol=1e-6)
    assert e["tw_rel_median"] == 0.0 and e["faces_equal"] == 0.9 and e["status_equal"] == 1.0 and e["n"] == n


def test_loss_masked():
    Q = np.array([10.0, 100.0, 5.0])
    Qt = np.array([1.0, 10.0, 5.0])
    Tw, Twt = np.array([1.0, 0.0, 2.0]), np.array([0.0, 0.0, 0.0])
    mask = np.array([True, True, False])
    # ((1)^2 + 0.1 * 1) and (1^2 + 0): mean 1.05
    assert math.isclose(bench.loss_masked(Q, Tw, Qt, Twt, mask), 1.05)


def test_job_rate_single_process():
    ms, rate = bench.job_rate(2.0, 1000)
    assert ms == 2.0 and math.isclose(rate, 1000 / 2e-3)


def _fake_smi(tmp_path, line):
    """An executable that prints ``line`` every -lms milliseconds, as
    nvidia-smi's query loop does."""
    p = tmp_path / "fake-smi"
    p.write_text("#!%s\n" % sys.executable + "import sys, time\n"
                 "ms = int(sys.argv[sys.argv.index('-lms') + 1])\n"
                 "while True:\n"
                 "    print(%r, flush=True)\n"
                 "    time.sleep(ms / 1000.0)\n" % line)
    p.chmod(0o755)
    return str(p)


def test_clock_sampler_keeps_the_samples_of_the_region(tmp_path):
    smi = _fake_smi(tmp_path, "0, 1980, 2070, 412.5, 0x4, Not Active, Not Active, Not Active, Active")
    c = bench.ClockSampler(0, smi=smi)
    c.start()
    time.sleep(0.1)  # before the region: not counted
    c.mark()
    time.sleep(0.2)
    out = c.stop()
    assert out["sm_mhz"] == 1980.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert 3 <= out["samples"] <= 0.2 / (bench.ClockSampler.INTERVAL_MS / 1000.0) + 2
    assert "bracketing" not in out and 190 <= out["region_ms"] < 400


def test_clock_sampler_short_region_and_missing_tool(tmp_path):
    smi = _fake_smi(tmp_path, "0, 2070, 2070, 300.0, 0x0, Not Active, Active, Not Active, Not Active")
    c = bench.ClockSampler(0, smi=smi)
    c.start()
    out = c.stop()  # a region shorter than the interval: the samples around it stand in
    assert out["samples"] == 0 and out["bracketing"] >= 1
    assert out["sm_mhz"] == 2070.0 and out["reasons"] == ["hw_thermal_slowdown"]
    c = bench.ClockSampler(0, smi=str(tmp_path / "absent"))
    c.start()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
