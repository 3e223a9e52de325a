"""bench.py's reference arm (the oracle on the host cores) prints one JSON
line with the contract's keys, on a small R-MAT so it runs without a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--scale", "12", "--steps", "4", "--warmup", "1"],
                         check=True, capture_output=True, text=True, cwd=ROOT, timeout=600).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["steps"] == 4 and d["warmup"] == 1
    assert d["unit"] == "GTEPS" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"] == {"value": d["value"], "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the timed steps take the step's algorithms in turn, so four steps sample all four
    assert sorted(d["cpu_baseline"]["per_algo"]) == ["bfs", "cc", "pagerank", "sssp"]
    assert all(p["steps"] == 1 and p["gteps"] > 0 for p in d["cpu_baseline"]["per_algo"].values())
    cfg = d["config"]
    assert cfg["workload"].startswith("rmat12 ") and cfg["V"] == 4096 and cfg["E"] == 65536
