"""Host logic of the serving loop (no GPU): the Poisson request generator,
the latency statistics, and the continuous-batching loop against a fake of
the serving calls."""
import numpy as np
import pytest

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


class _FakeServeLib:
    """Stands in for the serving calls of the C ABI: a query admitted with
    source s converges after (s % 5) + 1 steps of its engine; the result is
    the source repeated (so each retired query can be checked)."""

    def __init__(self):
        self.ctx = {}

    def begin(self, ctx, algo, slots):
        self.ctx[ctx] = {"slots": slots, "busy": {}, "steps": 0, "open": True}

    def admit(self, ctx, slot, source):
        c = self.ctx[ctx]
        assert c["open"] and slot not in c["busy"] and 0 <= slot < c["slots"]
        c["busy"][slot] = [source, (source % 5) + 1]

    def step(self, ctx):
        c = self.ctx[ctx]
        c["steps"] += 1
        fin = 0
        for slot, q in c["busy"].items():
            q[1] -= 1
            if q[1] == 0:
                fin |= 1 << slot
        busy = sum(1 << s for s in c["busy"])
        return fin, busy

    def fetch(self, ctx, slot, V, algo):
        src, left = self.ctx[ctx]["busy"].pop(slot)
        assert left == 0
        return np.full(V, src, np.uint32)

    def end(self, ctx):
        self.ctx[ctx]["open"] = False


@pytest.mark.parametrize("threads", [False, True])
def test_continuous_batching_loop(monkeypatch, threads):
    from paper_2208_14935_gb300 import hytg
    from paper_2208_14935_gb300.serve import Server

    lib = _FakeServeLib()
    monkeypatch.setattr(hytg, "hytg_serve_begin", lib.begin)
    monkeypatch.setattr(hytg, "hytg_serve_admit", lib.admit)
    monkeypatch.setattr(hytg, "hytg_serve_step", lib.step)
    monkeypatch.setattr(hytg, "hytg_serve_fetch", lib.fetch)
    monkeypatch.setattr(hytg, "hytg_serve_end", lib.end)

    class Eng:
        def __init__(self, name):
            self.ctx = name
            self.V = 8

    engines = {"bfs": Eng("b"), "sssp": Eng("s"), "ppr": Eng("p")}
    srv = Server(engines, slots={"bfs": 3, "sssp": 2, "ppr": 1}, threads=threads)
    pools = {"bfs": np.arange(0, 40), "sssp": np.arange(40, 80), "ppr": np.arange(80, 120)}
    reqs = poisson_requests(60, float("inf"), pools, seed=2)     # all at t = 0: slots bound admission
    done = srv.run(reqs)
    assert sorted(r.rid for r in done) == list(range(60))         # every query retired once
    for r in done:
        assert np.all(r.result == r.source)                        # its own slot's result
        assert r.arrival <= r.admitted <= r.done
    assert all(not c["open"] and not c["busy"] for c in lib.ctx.values())
    # each engine stepped only while it had work, and never more than its
    # queries' total steps (batching shares steps between queries)
    for name, algo in (("b", "bfs"), ("s", "sssp"), ("p", "ppr")):
        total = sum((r.source % 5) + 1 for r in reqs if r.algo == algo)
        assert 0 < lib.ctx[name]["steps"] <= total
    # the single-slot engine runs its queries one after another
    ppr = [r.source for r in reqs if r.algo == "ppr"]
    assert lib.ctx["p"]["steps"] == sum((s % 5) + 1 for s in ppr)


def test_threaded_loop_with_arrivals_over_time(monkeypatch):
    """Arrivals spread over time: every query is admitted after it arrives and
    retired once, with one host thread per engine."""
    from paper_2208_14935_gb300 import hytg
    from paper_2208_14935_gb300.serve import Server

    lib = _FakeServeLib()
    for name in ("begin", "admit", "step", "fetch", "end"):
        monkeypatch.setattr(hytg, f"hytg_serve_{name}", getattr(lib, name))

    class Eng:
        def __init__(self, name):
            self.ctx = name
            self.V = 4

    srv = Server({"bfs": Eng("b"), "ppr": Eng("p")}, slots={"bfs": 2, "ppr": 2}, threads=True)
    pools = {"bfs": np.arange(0, 10), "sssp": np.arange(0, 10), "ppr": np.arange(10, 20)}
    reqs = poisson_requests(40, 2000.0, pools, mix=(("bfs", 1), ("ppr", 1)), seed=4)
    done = srv.run(reqs)
    assert sorted(r.rid for r in done) == list(range(40))
    for r in done:
        assert r.admitted >= r.arrival and r.done >= r.admitted
        assert np.all(r.result == r.source)
