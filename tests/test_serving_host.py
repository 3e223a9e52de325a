"""Host logic of the serving loop (no GPU): the Poisson request generator."""
import numpy as np

from paper_2208_14935_gb300.serve import poisson_requests, Request, latency_stats


def test_poisson_requests():
    pools = {"bfs": np.arange(10), "sssp": np.arange(10, 20), "ppr": np.arange(20, 30)}
    reqs = poisson_requests(5000, 100.0, pools, seed=1)
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) >= 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 0.01) < 0.001                      # mean inter-arrival 1 / rate
    frac = {a: np.mean([r.algo == a for r in reqs]) for a in pools}
    assert abs(frac["bfs"] - 0.4) < 0.03 and abs(frac["ppr"] - 0.2) < 0.03
    for r in reqs:
        assert r.source in pools[r.algo]
    burst = poisson_requests(10, float("inf"), pools)
    assert all(r.arrival == 0.0 for r in burst)
    assert poisson_requests(50, 10.0, pools, seed=3)[7].source == poisson_requests(50, 10.0, pools, seed=3)[7].source


def test_latency_stats():
    done = [Request(i, 0.0, "bfs", 0, 0.0, 0.001 * (i + 1)) for i in range(100)]
    st = latency_stats(done)
    assert st["n"] == 100 and abs(st["p50_ms"] - 50.5) < 1e-6 and st["p99_ms"] > 99
