"""Device-driven iterations: single-source runs replay one iteration
(planning, binning, cache and zero-copy relax) inside a CUDA graph with a
WHILE node and return to the host only for iterations that need the F or C
route.  Results must equal the oracle's exactly (PageRank/PPR within 1e-4 L1)
with the loop on and off, and the per-iteration records and totals must
describe the same run."""
import numpy as np
import pytest

from gen import graphgen as gg
from oracle import oracle as orc

from test_gpu_parity import check, edge_bytes, engine, hy, rmat16, rmat16_sym  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("algo", ["bfs", "sssp", "cc", "pagerank", "ppr"])
@pytest.mark.parametrize("force", [-1, 4, 1])
def test_device_loop_routes(hy, rmat16, rmat16_sym, algo, force):
    g = rmat16_sym if algo == "cc" else rmat16
    budget = edge_bytes(g, algo) * 2 if force == 1 else edge_bytes(g, algo) // 4
    src = {"bfs": 0, "sssp": 0, "ppr": 5}.get(algo)
    runs = {}
    for loop in (0, 1):
        e = engine(hy, g, budget, force_route=force, device_loop=loop)
        got = e.run(algo, src)
        check(g, algo, got, 0 if src is None else src)
        runs[loop] = (got, e.stats(), e.iterations())
        e.close()
    st0, st1 = runs[0][1], runs[1][1]
    assert st0["graph_launches"] == 0
    if force == 4:                         # zero-copy only: every later iteration on the device
        assert st1["graph_iterations"] > 0
    if algo in ("bfs", "sssp", "cc"):
        assert np.array_equal(runs[0][0], runs[1][0])
    if algo in ("bfs", "sssp"):
        # activation is deterministic for min-updates (a vertex is activated
        # iff its smallest push beats its value at the start of the
        # iteration); CC's pointer jumping reads labels while they change
        assert st0["iterations"] == st1["iterations"]
        assert st0["edges_relaxed"] == st1["edges_relaxed"]
        assert st0["route_partitions"] == st1["route_partitions"]
        assert [r["active_edges"] for r in runs[0][2]] == [r["active_edges"] for r in runs[1][2]]
    its = runs[1][2]
    assert sum(r["active_edges"] for r in its) == st1["edges_relaxed"]


def test_device_loop_mesh(hy):
    """High diameter: hundreds of tiny-frontier iterations, buckets for SSSP."""
    g = gg.mesh(300, 200, shortcut_frac=0.001, radius=16, wmax=1000)
    s_on = {}
    for loop in (0, 1):
        e = engine(hy, g, g.E * 8 // 5, part_bytes=16384, device_loop=loop)
        for algo in ("bfs", "sssp", "cc"):
            got = e.run(algo, None if algo == "cc" else 0)
            check(g, algo, got, 0)
            s_on[(loop, algo)] = e.stats()
        e.close()
    for algo in ("bfs", "sssp", "cc"):
        a, b = s_on[(0, algo)], s_on[(1, algo)]
        if algo != "cc":
            assert a["iterations"] == b["iterations"], algo
            assert a["edges_relaxed"] == b["edges_relaxed"], algo
        assert b["graph_iterations"] > 0, algo


@pytest.mark.parametrize("delta", [1, 50, 0])
def test_device_loop_sssp_buckets(hy, delta):
    g = gg.mesh(120, 90, shortcut_frac=0.002, radius=8, wmax=1000, seed=3)
    e = engine(hy, g, g.E * 8 // 4, part_bytes=8192, sssp_delta=delta, force_route=4)
    check(g, "sssp", e.run("sssp", 0), 0)
    assert e.stats()["graph_iterations"] > 0
    e.close()


def test_device_loop_max_iters(hy, rmat16):
    outs = []
    for loop in (0, 1):
        e = engine(hy, rmat16, edge_bytes(rmat16, "bfs") // 4, force_route=4, max_iters=3, device_loop=loop)
        outs.append(e.run("bfs", 0))
        assert e.stats()["iterations"] == 3
        e.close()
    assert np.array_equal(outs[0], outs[1])
    want, _ = orc.bfs(rmat16, 0)
    reached = outs[1] != 0xFFFFFFFF
    assert np.array_equal(outs[1][reached], want[reached])
    assert outs[1][reached].max() <= 3


def test_device_loop_reuse_and_invalidation(hy, rmat16):
    """The captured graph is reused across runs and rebuilt when a parameter
    or the budget it depends on changes."""
    e = engine(hy, rmat16, edge_bytes(rmat16, "sssp") // 4)
    for algo in ("bfs", "sssp", "bfs", "pagerank", "bfs"):
        check(rmat16, algo, e.run(algo, None if algo == "pagerank" else 0), 0)
    e.set_param("alpha", 0.6)
    check(rmat16, "bfs", e.run("bfs", 0), 0)
    e.set_budget(edge_bytes(rmat16, "sssp") // 3)
    check(rmat16, "sssp", e.run("sssp", 0), 0)
    e.set_param("part_bytes", 32 * 1024)
    check(rmat16, "bfs", e.run("bfs", 0), 0)
    e.close()


def test_device_loop_param(hy, rmat16):
    e = engine(hy, rmat16, rmat16.E)
    assert e.get_param("device_loop") == 1
    e.set_param("device_loop", 2)
    with pytest.raises(hy.HytgError):
        e.set_param("device_loop", 3)
    e.close()


@pytest.mark.parametrize("algo", ["bfs", "sssp", "cc", "pagerank", "ppr"])
@pytest.mark.parametrize("force", [-1, 2, 3])
def test_device_loop_f_and_c(hy, rmat16, rmat16_sym, algo, force):
    """device_loop 2: iterations that send partitions to F (each copied into a
    staging slot by its IF node, then relaxed) or C (gathered and relaxed by
    the C node) stay in the graph; results equal the oracle and the host loop."""
    g = rmat16_sym if algo == "cc" else rmat16
    src = {"bfs": 0, "sssp": 0, "ppr": 5}.get(algo)
    e = engine(hy, g, edge_bytes(g, algo) // 4, force_route=force, device_loop=2)
    got = e.run(algo, src)
    check(g, algo, got, 0 if src is None else src)
    st = e.stats()
    its = e.iterations()
    assert sum(r["active_edges"] for r in its) == st["edges_relaxed"]
    if force == 2:
        # every iteration after the first (run before the graph is captured)
        assert st["graph_iterations"] == st["iterations"] - 1 and st["f_tasks"] > 0
        assert st["link_bytes"][2] > 0
    elif force == -1:
        assert st["graph_iterations"] > 0
    e.set_param("device_loop", 0)
    got0 = e.run(algo, src)
    if algo in ("bfs", "sssp", "cc"):
        assert np.array_equal(got0, got)
    e.close()


@pytest.mark.parametrize("algo,k", [("bfs", 64), ("sssp", 64), ("ppr", 32)])
@pytest.mark.parametrize("force", [-1, 4])
def test_device_loop_batched(hy, rmat16, algo, k, force):
    """Batched runs in the device loop: the per-iteration source commit takes
    its level from the control block."""
    rng = np.random.default_rng(11)
    cand = np.flatnonzero(np.diff(rmat16.off.astype(np.int64)) > 0)
    src = [0] + rng.choice(cand, k - 1, replace=False).tolist()
    e = engine(hy, rmat16, edge_bytes(rmat16, algo) // 4, force_route=force, device_loop=1)
    got = e.run(algo, src)
    st = e.stats()
    if force == 4:
        assert st["graph_iterations"] > 0
    if force == -1:
        # F and C iterations stay in the graph for batched runs
        assert st["graph_iterations"] >= st["iterations"] // 2 > 0, st
    for s, v in enumerate(src[:8] + src[-4:]):
        row = got[src.index(v)]
        if algo == "bfs":
            assert np.array_equal(row, orc.bfs(rmat16, v)[0]), f"source {v}"
        elif algo == "sssp":
            assert np.array_equal(row, orc.sssp(rmat16, v)[0]), f"source {v}"
        else:
            x, _, _ = orc.pagerank(rmat16, tol=1e-13, seed=v)
            assert float(np.abs(row.astype(np.float64) - x).sum()) <= 1e-4, f"seed {v}"
    e.set_param("device_loop", 0)
    got0 = e.run(algo, src)
    if algo != "ppr":
        assert np.array_equal(got0, got)
    e.close()


@pytest.mark.parametrize("loop", [0, 1])
def test_run_deadline(hy, loop):
    """A run past "run_timeout_ms" stops at an iteration boundary with
    HYTG_ERR_TIMEOUT (inside the device loop through the cancel word the host
    sets, on the host loop before the next iteration), leaves no result, and
    the same context then runs to the exact result without a deadline."""
    g = gg.mesh(1024, 1024, shortcut_frac=0.0, wmax=1000)     # BFS: 2,047 iterations
    e = engine(hy, g, g.E * 16, part_bytes=1 << 20, device_loop=loop)   # all cached
    e.set_param("run_timeout_ms", 3)
    with pytest.raises(hy.HytgError) as ex:
        e.run("bfs", 0)
    assert ex.value.status == hy.HYTG_ERR_TIMEOUT
    st = e.stats()
    assert 0 < st["iterations"] < 2047
    with pytest.raises(hy.HytgError) as ex:
        hy.hytg_fetch_result(e.ctx, g.V, hy.HYTG_BFS)
    assert ex.value.status == hy.HYTG_ERR_STATE
    e.set_param("run_timeout_ms", 0)
    got = e.run("bfs", 0)
    check(g, "bfs", got, 0)
    assert e.stats()["iterations"] >= 2047
    if loop:
        assert e.stats()["graph_iterations"] > 0
    e.set_param("run_timeout_ms", 60000)         # a deadline far away changes nothing
    assert np.array_equal(e.run("bfs", 0), got)
    e.close()


@pytest.mark.parametrize("algo", ["bfs", "sssp", "pagerank"])
def test_loop_after_fc(hy, rmat16, algo):
    """Whether the host plans PageRank's iteration after one with F or C
    work ("loop_after_fc" 0, the default) or the device loop takes over after
    every host iteration (1), the results are the same, and for BFS/SSSP
    (which always take the device loop) so are the iterations and the edges
    relaxed; the mesh still runs iterations in the graph."""
    src = None if algo == "pagerank" else 0
    runs = {}
    for v in (0, 1):
        e = engine(hy, rmat16, edge_bytes(rmat16, algo) // 4, loop_after_fc=v)
        assert e.get_param("loop_after_fc") == v
        got = e.run(algo, src)
        check(rmat16, algo, got, 0)
        runs[v] = (got, e.stats())
        e.close()
    if algo != "pagerank":
        assert np.array_equal(runs[0][0], runs[1][0])
        assert runs[0][1]["iterations"] == runs[1][1]["iterations"]
        assert runs[0][1]["edges_relaxed"] == runs[1][1]["edges_relaxed"]
    g = gg.mesh(200, 100, shortcut_frac=0.001, radius=8, wmax=1000)
    if algo != "pagerank":
        e = engine(hy, g, g.E * 8 // 5, part_bytes=16384)
        check(g, algo, e.run(algo, 0), 0)
        st = e.stats()
        assert st["graph_iterations"] > 0, st
        e.close()
