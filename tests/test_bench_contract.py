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


def test_copy_boundaries():
    """The copy engine's busy time is the union of the copy intervals, and
    idle stretches are counted only past the threshold."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    dt = np.dtype([("kind", np.uint32), ("start_ms", np.float64), ("end_ms", np.float64)])
    rows = [(8, 0.0, 1.0), (8, 0.5, 1.5), (4, 1.0, 3.0), (8, 1.52, 2.0),   # back to back
            (8, 2.6, 3.0), (7, 3.0, 3.1), (8, 3.05, 4.0), (8, 4.3, 5.0)]   # gaps 0.6, 0.05, 0.3
    tl = np.array(rows, dtype=dt)
    r = bench.copy_boundaries(tl, min_gap_ms=0.1)
    assert abs(r["copy_busy_ms"] - (1.5 + 0.48 + 0.4 + 0.95 + 0.7)) < 1e-9
    assert r["idle_stretches"] == 2 and abs(r["idle_stretch_ms"] - 0.45) < 1e-9
    assert bench.copy_boundaries(tl[:2])["idle_stretch_ms"] is None
    assert bench.union_ms([(0, 2), (1, 3), (5, 6)]) == 4
