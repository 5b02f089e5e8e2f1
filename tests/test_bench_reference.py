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


def test_stated_error_helpers():
    """The bench's per-output errors: per probe trace (rows), per snapshot (columns), and
    the functional scale max |dy| / (||C_p|| max ||I||), checked on hand-made arrays."""
    import numpy as np
    import bench
    ref = np.array([[3.0, 4.0], [1e-6, 0.0]])          # two probe traces
    got = ref + np.array([[0.0, 5e-3], [1e-8, 0.0]])
    # trace 0: 5e-3 / 5 = 1e-3; trace 1: 1e-8 / 1e-6 = 1e-2 -> the small trace decides
    assert abs(bench._per_trace(got, ref) - 1e-2) < 1e-12
    snaps = np.array([[1.0, 0.0], [0.0, 2.0]])          # two snapshots (columns)
    s2 = snaps + np.array([[1e-3, 0.0], [0.0, 0.0]])
    assert abs(bench._per_snapshot(s2, snaps) - 1e-3) < 1e-15
    assert bench._per_snapshot(np.zeros((2, 0)), np.zeros((2, 0))) is None
    C = np.array([[2.0, 0.0], [0.0, 1.0]])
    # max |dy| per probe: 5e-3 and 1e-8; ||C_p|| = 2 and 1; max ||I|| = 2: on this scale
    # the small trace's error is negligible
    f = bench._functional(got, ref, C, snaps)
    assert abs(f - max(5e-3 / (2 * 2), 1e-8 / (1 * 2))) < 1e-15


def test_snapshot_view():
    """The modal snapshot product's rate from the chunk time outside the scan: bytes of
    U's kept slices (16 n0^2 per group of up to 32 columns) over (run - scan) per chunk;
    none below the kept-slice size or without snapshots."""
    import bench
    # 10 chunks, 130 ms run, 30 ms scan -> 10 ms per chunk; n0 = 8192, 4 snapshots:
    # 16 * 8192^2 B = 1.073741824 GB in 10 ms = 107.3741824 GB/s
    v = bench._snapshot_view(130.0, 30.0, 10, 8192, 4, 1000.0)
    assert abs(v["ms_per_chunk_outside_scan"] - 10.0) < 1e-12
    assert abs(v["achieved_lower_bound"] - 107.3741824) < 1e-9
    assert abs(v["frac_lower_bound"] - 0.1073741824) < 1e-12
    # 33 snapshots are two column groups: twice the bytes, twice the rate
    v2 = bench._snapshot_view(130.0, 30.0, 10, 8192, 33, 1000.0)
    assert abs(v2["achieved_lower_bound"] - 2 * 107.3741824) < 1e-9
    assert bench._snapshot_view(130.0, 30.0, 10, 4095, 4, 1000.0) is None
    assert bench._snapshot_view(130.0, 30.0, 10, 8192, 0, 1000.0) is None
    assert bench._snapshot_view(30.0, 30.0, 10, 8192, 4, 1000.0) is None
