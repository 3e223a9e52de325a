"""Serving with continuous batching: queries that arrive while others are on
the GPU join the running batch at the next iteration, slots are reused as
queries finish, and every result equals the query's result alone (BFS/SSSP
bit-exact against the oracle and the single-query run; PPR within 1e-4 L1)."""
import numpy as np
import pytest

from gen import graphgen as gg
from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hy():
    from paper_2208_14935_gb300 import build, hytg
    build.build()
    hytg.load()
    return hytg


@pytest.fixture(scope="module")
def g():
    return gg.rmat(15, seed=4)


@pytest.fixture(scope="module")
def engines(hy, g):
    unweighted = gg.CSR(g.V, g.E, g.off, g.dst, None)
    out = {}
    for algo in ("bfs", "sssp", "ppr"):
        e = hy.Engine(params={"part_bytes": 32 * 1024})
        e.load(g if algo == "sssp" else unweighted)
        e.set_budget(g.E * (8 if algo == "sssp" else 4) // 4)
        out[algo] = e
    yield out
    for e in out.values():
        e.close()


def check(g, r, tol=1e-4):
    if r.algo == "bfs":
        assert np.array_equal(r.result, orc.bfs(g, r.source)[0]), r
    elif r.algo == "sssp":
        assert np.array_equal(r.result, orc.sssp(g, r.source)[0]), r
    else:
        x, _, _ = orc.pagerank(g, tol=1e-13, seed=r.source)
        assert float(np.abs(r.result.astype(np.float64) - x).sum()) <= tol, r


def test_join_mid_run(hy, g, engines):
    """Admit A, step twice, admit B into the running batch; both are exact."""
    e = engines["bfs"]
    hy.hytg_serve_begin(e.ctx, hy.HYTG_BFS, 4)
    hy.hytg_serve_admit(e.ctx, 0, 0)
    for _ in range(2):
        hy.hytg_serve_step(e.ctx)
    hy.hytg_serve_admit(e.ctx, 2, 123)
    got = {}
    for _ in range(200):
        fin, busy = hy.hytg_serve_step(e.ctx)
        for s in (0, 2):
            if fin >> s & 1:
                got[s] = hy.hytg_serve_fetch(e.ctx, s, g.V, hy.HYTG_BFS)
        if len(got) == 2:
            break
    hy.hytg_serve_end(e.ctx)
    assert np.array_equal(got[0], orc.bfs(g, 0)[0])
    assert np.array_equal(got[2], orc.bfs(g, 123)[0])


def test_mixed_stream_same_alone_and_in_mix(hy, g, engines):
    from paper_2208_14935_gb300.serve import Server, poisson_requests, latency_stats
    cand = np.flatnonzero(np.diff(g.off.astype(np.int64)) > 0)
    rng = np.random.default_rng(0)
    pools = {a: rng.choice(cand, 64) for a in ("bfs", "sssp", "ppr")}
    reqs = poisson_requests(60, 2000.0, pools, seed=5)         # arrivals overlap running queries
    srv = Server(engines, slots={"bfs": 6, "sssp": 6, "ppr": 3})   # fewer slots than queries
    done = srv.run(reqs)
    assert len(done) == len(reqs)
    assert {r.algo for r in done} == {"bfs", "sssp", "ppr"}
    for r in done:
        assert r.done >= r.admitted >= r.arrival >= 0
        check(g, r)
    # alone: the same queries, one at a time, through the single-query path
    for r in done[:12]:
        alone = engines[r.algo].run(r.algo, r.source)
        if r.algo == "ppr":
            assert float(np.abs(alone.astype(np.float64) - r.result).sum()) <= 1e-4
        else:
            assert np.array_equal(alone, r.result)
    st = latency_stats(done)
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_serving_errors(hy, g, engines):
    e = engines["sssp"]
    with pytest.raises(hy.HytgError):
        hy.hytg_serve_step(e.ctx)                      # not serving
    hy.hytg_serve_begin(e.ctx, hy.HYTG_SSSP, 2)
    hy.hytg_serve_admit(e.ctx, 0, 1)
    with pytest.raises(hy.HytgError):
        hy.hytg_serve_admit(e.ctx, 0, 2)               # busy slot
    with pytest.raises(hy.HytgError):
        hy.hytg_serve_admit(e.ctx, 2, 2)               # slot out of range
    with pytest.raises(hy.HytgError):
        hy.hytg_run(e.ctx, hy.HYTG_SSSP, [0])          # single runs wait for serve_end
    fin = 0
    while not fin & 1:
        fin, _ = hy.hytg_serve_step(e.ctx)
    d = hy.hytg_serve_fetch(e.ctx, 0, g.V, hy.HYTG_SSSP)
    with pytest.raises(hy.HytgError):
        hy.hytg_serve_fetch(e.ctx, 0, g.V, hy.HYTG_SSSP)   # already fetched
    hy.hytg_serve_end(e.ctx)
    assert np.array_equal(d, orc.sssp(g, 1)[0])
