"""The CPU-compaction form of ExpTM-C (Sec. III-B; "compact_host" = n host
threads): the C route's active lists are compacted on the host into pinned
staging chunks and copied in with one explicit copy per chunk.  Results must
equal the oracle's exactly as with the GPU gather (BFS/SSSP/CC bit-exact,
PageRank/PPR within 1e-4 L1), for one and several threads, with the route
spread over many staging chunks, and in batched runs."""
import numpy as np
import pytest

from gen import graphgen as gg
from oracle import oracle as orc

from test_gpu_parity import check, edge_bytes, engine, hy, rmat16, rmat16_sym  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("algo", ["bfs", "sssp", "cc", "pagerank", "ppr"])
@pytest.mark.parametrize("threads", [1, 4])
@pytest.mark.parametrize("force", [3, 5])
def test_host_compaction_routes(hy, rmat16, rmat16_sym, algo, threads, force):
    g = rmat16_sym if algo == "cc" else rmat16
    e = engine(hy, g, edge_bytes(g, algo) // 4, force_route=force, compact_host=threads, seed=9)
    src = {"bfs": 0, "sssp": 0, "ppr": 5}.get(algo)
    check(g, algo, e.run(algo, src), 0 if src is None else src)
    st = e.stats()
    assert st["route_partitions"][3] > 0
    assert st["host_compact_ms"] > 0
    ebytes = 8 if algo == "sssp" else 4
    assert st["link_bytes"][3] == st["route_edges"][3] * ebytes + st["route_vertices"][3] * 16
    e.close()


@pytest.mark.parametrize("algo", ["bfs", "sssp", "pagerank"])
def test_host_compaction_many_chunks(hy, rmat16, algo):
    """Compaction buffer at its 2048-edge minimum: every C iteration spans
    many chunks, alternating between the two pinned staging buffers."""
    e = engine(hy, rmat16, edge_bytes(rmat16, "sssp") // 4, force_route=3, compact_host=3,
               compact_frac=0.001)
    src = None if algo == "pagerank" else 0
    check(rmat16, algo, e.run(algo, src), 0)
    assert e.info()["compact_edges"] == 2048
    its = e.iterations()
    assert max(r["route_edges"][3] for r in its) > 8 * 2048
    e.close()


def test_host_compaction_matches_gpu_gather(hy, rmat16):
    """Same routes, same results and the same per-iteration active edges
    whichever side compacts."""
    runs = {}
    for threads in (0, 2):
        e = engine(hy, rmat16, edge_bytes(rmat16, "sssp") // 4, compact_host=threads)
        d = e.run("sssp", 0)
        runs[threads] = (d, [r["route_edges"] for r in e.iterations()], e.stats())
        e.close()
    assert np.array_equal(runs[0][0], runs[2][0])
    assert runs[0][1] == runs[2][1]
    assert runs[0][2]["host_compact_ms"] == 0


def test_host_compaction_batched(hy, rmat16):
    rng = np.random.default_rng(4)
    cand = np.flatnonzero(np.diff(rmat16.off.astype(np.int64)) > 0)
    src = [0] + rng.choice(cand, 31, replace=False).tolist()
    e = engine(hy, rmat16, rmat16.E, force_route=3, compact_host=4)
    lv = e.run("bfs", src)
    for s, v in enumerate(src):
        assert np.array_equal(lv[s], orc.bfs(rmat16, v)[0]), f"source {s} ({v})"
    e.close()


@pytest.mark.parametrize("V,E", [(1, 0), (33, 200), (1000, 6000), (4097, 30000)])
def test_host_compaction_irregular(hy, V, E):
    g = gg.random_graph(V, E, seed=V + E, skew=1.1)
    e = engine(hy, g, max(64 * 1024, g.E * 2), force_route=3, part_bytes=4096, compact_host=5)
    for src in sorted({0, g.V - 1}):
        check(g, "bfs", e.run("bfs", src), src)
        check(g, "sssp", e.run("sssp", src), src)
    e.close()


def test_host_compaction_param(hy, rmat16):
    e = engine(hy, rmat16, rmat16.E)
    assert e.get_param("compact_host") == 0
    for bad in (-1, 1.5, 257):
        with pytest.raises(hy.HytgError):
            e.set_param("compact_host", bad)
    e.set_param("compact_host", 8)
    assert e.get_param("compact_host") == 8
    e.close()
