"""The per-run JSON-lines record written by ThetaMethod(log_path=...) (host logic only)."""
import json

from paper_2407_11993_gb300 import eddy


def test_append_run_record(tmp_path):
    path = tmp_path / "runs.jsonl"
    t = {"run_ms": 50.0, "run_steps": 20000, "setup_ms": 4500.0}
    eddy.append_run_record(str(path), {"form": "modal", "n": 8192, "T": 20000}, t)
    eddy.append_run_record(str(path), {"form": "plain", "n": 8192, "T": 10}, {"run_ms": 0.0})
    lines = path.read_text().splitlines()
    assert len(lines) == 2
    a, b = (json.loads(x) for x in lines)
    assert a["config"]["form"] == "modal" and a["timings"]["setup_ms"] == 4500.0
    assert abs(a["steps_per_s"] - 400000.0) < 1e-6
    assert b["steps_per_s"] is None
