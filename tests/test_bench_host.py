"""Host logic of bench.py on CPU: the clock summary, the roofline's traffic
scaling, the HBM peak lookup, and the reference arm's JSON line (the FP64
oracle timed on the host, one small step)."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_clock_summary_reads_median_max_and_active_reasons():
    c = bench.ClockSampler(0)
    c.proc = object()  # as if nvidia-smi had run
    c.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1980, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active\n",
        "0, 2070, 2070, 1300.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
        "garbage line\n",
    ]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_summary_without_a_sampler_is_none():
    with bench.ClockSampler(0) as c:
        pass
    if c.proc is None:
        assert c.summary() is None


def test_traffic_per_pixel_iteration_reproduces_the_captures():
    # the 64-pair captures: FP32 82,310,400 pixel-iterations, 3.477 + 0.189 GB;
    # FP16 83,980,800 pixel-iterations, 1.801 + 0.171 GB
    t = bench.NCU_TRAFFIC_PER_PX_ITER
    assert t[("k_icp_sched", "fp32")] * 82310400 == pytest.approx(3477426688 + 188985088, rel=1e-12)
    assert t[("k_icp_sched", "fp16")] * 83980800 == pytest.approx(1800692224 + 170857472, rel=1e-12)
    # one pass: about the 36 B (18 B) unit plus the window records, not the
    # 67 B of two passes
    assert 36.0 < t[("k_icp_sched", "fp32")] < 50.0
    assert 18.0 < t[("k_icp_sched", "fp16")] < 27.0


def test_traffic_entries_are_per_pixel_iteration_figures():
    # every stored figure is DRAM bytes per pixel-iteration of one launch: at
    # least the algorithmic unit of its precision, and not a per-launch total
    for (kern, prec), per_px in bench.NCU_TRAFFIC_PER_PX_ITER.items():
        unit = 18 if prec == "fp16" else 36
        assert kern == "k_icp_sched" and unit * 0.9 <= per_px < 4 * unit, (kern, prec, per_px)


def test_hbm_peak_comes_from_the_measured_file_when_present():
    peak, src = bench.hbm_peak()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            assert peak == float(json.load(f)["hbm_gbs"])
        assert src.startswith("measured")
    else:
        assert peak == 6800.0 and src.startswith("fallback")


def test_workload_name_states_the_pairs_and_precision():
    name = bench.workload_name(256, "fp32")
    assert "256 independent" in name and name.startswith("kinect-640x480-3level fp32")


@pytest.mark.slow
def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    d = json.loads(lines[-1])
    assert d["impl"] == "reference" and d["unit"] == "alignments/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["higher_is_better"] is True and d["steps"] == 1
