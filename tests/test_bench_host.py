"""Host logic of the benchmark (no GPU): the algorithmic byte model the FP32 roofline
divides by, the roofline arithmetic, the measured-traffic lookup keyed by the CUDA
sources' hash, the clock-scaled FP64 peak, the clock record's parsing and the FP32 error
measure."""
import json
import os

import numpy as np
import pytest

import bench


def test_byte_model_plane_counts():
    # plane-accesses per cell and step: explicit 10 + 18, right-hand side 6 + 8, three
    # transform passes of 2 + 2, update 12 + 20 (FP64) or 12 + 26 (FP32, the close writes
    # the populations and the next step's moments)
    f64 = bench.step_bytes_per_cell(False)
    f32 = bench.step_bytes_per_cell(True)
    assert {k: v // 8 for k, v in f64.items()} == {"explicit": 28, "rhs": 14, "fft_rows_fwd": 4, "fft_cols": 4,
                                                   "fft_rows_inv": 4, "update": 32}
    assert {k: v // 4 for k, v in f32.items()} == {"explicit": 28, "rhs": 14, "fft_rows_fwd": 4, "fft_cols": 4,
                                                   "fft_rows_inv": 4, "update": 38}
    assert sum(f32.values()) == 368                  # B per cell and step, the figure the design states


def test_flop_model_is_positive_and_grows_with_the_transform_length():
    a, b = bench.step_flops_per_cell("WENO5_C4", 1024), bench.step_flops_per_cell("WENO5_C4", 2048)
    assert all(v > 0 for v in a.values())
    assert b["fft_cols"] > a["fft_cols"] and b["explicit"] == a["explicit"]
    assert bench.step_flops_per_cell("LF1_C2", 2048)["explicit"] < b["explicit"]


def test_roofline_arithmetic():
    cells, steps = 2048 * 2048, 3
    # dominant kind: update, 2 launches per step of 0.25 ms each
    prof = {"explicit": (1.2, 6), "update": (1.5, 6), "rhs": (0.4, 6)}
    kind, r = bench.roofline(prof, steps, cells, True, "WENO5_C4", 2048, {"hbm_gbs": 6000.0})
    assert kind == "update" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    per_launch = bench.step_bytes_per_cell(True)["update"] * cells / 2
    assert r["algorithmic_bytes_per_launch"] == per_launch
    assert r["achieved"] == pytest.approx(per_launch / 0.25e-3 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0, rel=1e-3)
    # the FP64 form against the clock-scaled FMA peak
    kind, r = bench.roofline(prof, steps, cells, False, "WENO5_C4", 2048, {},
                             {"tflops_at_run_clock": 1.25, "source": "test"})
    flops = bench.step_flops_per_cell("WENO5_C4", 2048)["update"] * cells / 2
    assert r["bound"] == "alu" and r["achieved"] == pytest.approx(flops / 0.25e-3 / 1e12, rel=1e-3)


def test_scaled_peak_follows_the_clock():
    leg = {"tflops": 1.25, "clocks": {"sm_mhz": 2070.0}}
    assert bench.scaled_peak(leg, {"sm_mhz": 1035.0})["tflops_at_run_clock"] == pytest.approx(0.625)
    assert bench.scaled_peak(leg, {"sm_mhz": None})["tflops_at_run_clock"] == pytest.approx(1.25)


def test_measured_traffic_only_for_the_recorded_sources(tmp_path, monkeypatch):
    rec = {"n": 2048, "csrc_sha256": bench.csrc_digest(), "fp32": {"update": 123.0}, "fp64": {"explicit": 456.0}}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    assert bench.measured_traffic("update", True, 2048) == 123.0
    assert bench.measured_traffic("explicit", False, 2048) == 456.0
    assert bench.measured_traffic("update", True, 1024) is None          # another size
    rec["csrc_sha256"] = "0" * 64                                       # other kernels
    path.write_text(json.dumps(rec))
    assert bench.measured_traffic("update", True, 2048) is None


def test_clock_record_parsing(tmp_path):
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "clk.csv")
    with open(c.path, "w") as f:
        f.write("0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 2070, 2070, 950.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 1900, 2070, 990.0, 0x4, Not Active, Not Active, Not Active, Active\n")
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(c.path)


def test_fp32_error_measure():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((6, 16, 16))
    assert bench.fp32_errors(X, X) == (0.0, 0.0)
    Y = X.copy()
    Y[0] += 1e-6 * np.max(np.hypot(X[0], X[1]))
    vel, _ = bench.fp32_errors(Y, X)
    assert vel == pytest.approx(1e-6, rel=1e-6)


def test_l2_note_follows_the_size():
    assert bench.l2_note(2048) == "inputs larger than L2 (FP64 state 201 MB, step working set ~1.7 GB)"
    assert bench.l2_note(512).startswith("inputs smaller than L2")


def test_reference_arm_line():
    # the oracle on the host cores, small grid: the line the contract asks for, impl reference
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(os.path.dirname(bench.__file__), "bench.py"), "--impl", "reference",
                        "--n", "32", "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["grid"] == [32, 32] and "smaller than L2" in line["config"]["l2"]
