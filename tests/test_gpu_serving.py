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
        # a quarter of the edge bytes for the edge side, plus the query
        # frames of every slot (8 queries each: V * 32 B, PPR V * 96 B)
        frames = 4 * g.V * 96 if algo == "ppr" else 8 * g.V * 32
        e.set_budget(g.E * (8 if algo == "sssp" else 4) // 4 + frames + (1 << 16))
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


def _one_frame_engine(hy, g):
    """A BFS engine whose budget holds a quarter of the edge bytes and one
    frame of query state (8 queries) beside them."""
    e = hy.Engine(params={"part_bytes": 32 * 1024})
    e.load(gg.CSR(g.V, g.E, g.off, g.dst, None))
    e.set_budget(g.E * 4 // 4 + g.V * 32 + (1 << 16))
    return e


def test_query_waits_for_memory_not_a_slot(hy, g):
    """With 64 slots but memory for 8 queries, the ninth is refused for
    memory although its slot is free (HYTG_ERR_BUDGET, nothing admitted);
    once the first group's queries are fetched their frame is free again and
    the ninth runs; every result is exact."""
    e = _one_frame_engine(hy, g)
    hy.hytg_serve_begin(e.ctx, hy.HYTG_BFS, 64)
    info = hy.hytg_serve_get_info(e.ctx)
    assert info["frames"] == 1 and info["frames_free"] == 1 and info["slots_per_frame"] == 8
    assert info["frame_bytes"] >= g.V * 32
    srcs = [int(x) for x in np.flatnonzero(np.diff(g.off.astype(np.int64)) > 0)[:9 * 50:50]]
    for s in range(8):
        hy.hytg_serve_admit(e.ctx, s, srcs[s])
    assert hy.hytg_serve_get_info(e.ctx)["frames_free"] == 0
    with pytest.raises(hy.HytgError) as ex:
        hy.hytg_serve_admit(e.ctx, 8, srcs[8])            # free slot, no free memory
    assert ex.value.status == hy.HYTG_ERR_BUDGET
    assert hy.hytg_serve_get_info(e.ctx)["busy_slots"] == 0xFF
    got = {}
    for _ in range(500):
        fin, _ = hy.hytg_serve_step(e.ctx)
        for s in range(8):
            if fin >> s & 1:
                got[s] = hy.hytg_serve_fetch(e.ctx, s, g.V, hy.HYTG_BFS)
                if len(got) < 8:
                    assert hy.hytg_serve_get_info(e.ctx)["frames_free"] == 0
        if len(got) == 8:
            break
    assert hy.hytg_serve_get_info(e.ctx)["frames_free"] == 1
    hy.hytg_serve_admit(e.ctx, 8, srcs[8])
    for _ in range(500):
        fin, _ = hy.hytg_serve_step(e.ctx)
        if fin >> 8 & 1:
            got[8] = hy.hytg_serve_fetch(e.ctx, 8, g.V, hy.HYTG_BFS)
            break
    hy.hytg_serve_end(e.ctx)
    e.close()
    for s in range(9):
        assert np.array_equal(got[s], orc.bfs(g, srcs[s])[0]), s


@pytest.mark.parametrize("threads", [False, True])
def test_server_admits_by_memory(hy, g, threads):
    """A burst of 20 queries on an engine with 64 slots and memory for 8: the
    server keeps at most 8 on the device, the others wait for memory, and
    every result equals the query's result alone."""
    from paper_2208_14935_gb300.serve import Server, poisson_requests
    e = _one_frame_engine(hy, g)
    cand = np.flatnonzero(np.diff(g.off.astype(np.int64)) > 0)
    reqs = poisson_requests(20, float("inf"), {"bfs": cand[:200]}, mix=(("bfs", 1),), seed=2)
    srv = Server({"bfs": e}, slots={"bfs": 64}, threads=threads)
    done = srv.run(reqs)
    lane = srv.lanes["bfs"]
    assert len(done) == 20 and lane.max_busy == 8 and lane.memory_waits > 0
    for r in done:
        check(g, r)
    e.close()


def test_threaded_server_same_alone_and_in_mix(hy, g, engines):
    """The server with one host thread per engine: every retired query equals
    the oracle and its single-query run."""
    from paper_2208_14935_gb300.serve import Server, poisson_requests
    cand = np.flatnonzero(np.diff(g.off.astype(np.int64)) > 0)
    rng = np.random.default_rng(1)
    pools = {a: rng.choice(cand, 64) for a in ("bfs", "sssp", "ppr")}
    reqs = poisson_requests(45, 2000.0, pools, seed=6)
    srv = Server(engines, slots={"bfs": 16, "sssp": 16, "ppr": 8}, threads=True)
    done = srv.run(reqs)
    assert len(done) == len(reqs) and {r.algo for r in done} == {"bfs", "sssp", "ppr"}
    for r in done:
        assert r.done >= r.admitted >= r.arrival >= 0
        check(g, r)
    for r in done[:9]:
        alone = engines[r.algo].run(r.algo, r.source)
        if r.algo == "ppr":
            assert float(np.abs(alone.astype(np.float64) - r.result).sum()) <= 1e-4
        else:
            assert np.array_equal(alone, r.result)
