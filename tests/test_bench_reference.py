"""The reference arm of bench.py (the FP64 oracle timed on the host cores) keeps the JSON
line contract; runs on CPU at the smallest workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "n512_coil",
                        "--steps", "1", "--warmup", "0", "--oracle-steps", "3"],
                       capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    import bench
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC
    assert line["unit"] == "steps/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_clock_summary_reads_throttle_reasons():
    import bench
    lines = ["2070, 2070, 812.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "1980, 2070, 1391.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "2070, 2070, 900.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "garbage line", "N/A, 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = bench.ClockSampler.summarize(lines)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert bench.ClockSampler.summarize([])["sm_mhz"] is None
