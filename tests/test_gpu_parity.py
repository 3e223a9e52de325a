"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

BFS levels, SSSP distances and CC labels must be bit-exact; PageRank and
personalised PageRank within 1e-4 in L1 of the normalised vectors (the
tolerance the task sets for FP32 delta-PageRank against the FP64 oracle).
Every route is exercised alone (forced), at random per partition and
iteration, and under the cost model; results must not depend on the route.
"""
from fractions import Fraction

import numpy as np
import pytest

from gen import graphgen as gg
from oracle import oracle as orc
from oracle import planner as pl

pytestmark = pytest.mark.gpu

PR_TOL = 1e-4


@pytest.fixture(scope="module")
def hy():
    from paper_2208_14935_gb300 import build, hytg
    build.build()
    hytg.load()
    return hytg


@pytest.fixture(scope="module")
def rmat16():
    return gg.rmat(16, seed=1)


@pytest.fixture(scope="module")
def rmat16_sym(rmat16):
    return gg.symmetrize(rmat16)


def edge_bytes(g, algo):
    return g.E * (8 if algo == "sssp" else 4)


def engine(hy, g, budget, **params):
    e = hy.Engine(params={"part_bytes": 64 * 1024, **params})
    e.load(g)
    e.set_budget(int(budget))
    return e


def check(g, algo, got, src=0):
    if algo == "bfs":
        want, _ = orc.bfs(g, src)
        assert np.array_equal(got, want), f"BFS mismatch at {np.flatnonzero(got != want)[:10]}"
    elif algo == "sssp":
        want, _, _ = orc.sssp(g, src)
        assert np.array_equal(got, want), f"SSSP mismatch at {np.flatnonzero(got != want)[:10]}"
    elif algo == "cc":
        want = orc.cc(g)
        assert np.array_equal(got, want), f"CC mismatch at {np.flatnonzero(got != want)[:10]}"
    elif algo == "pagerank":
        x, _, _ = orc.pagerank(g, tol=1e-13)
        err = float(np.abs(got.astype(np.float64) - x).sum())
        assert err <= PR_TOL, f"PageRank L1 {err}"
        assert abs(float(got.astype(np.float64).sum()) - 1.0) < 1e-5
    elif algo == "ppr":
        x, _, _ = orc.pagerank(g, tol=1e-13, seed=src)
        err = float(np.abs(got.astype(np.float64) - x).sum())
        assert err <= PR_TOL, f"PPR L1 {err}"


FORCE = [-1, 2, 3, 4, 5]


@pytest.mark.parametrize("algo", ["bfs", "sssp", "pagerank", "ppr"])
@pytest.mark.parametrize("force", FORCE)
def test_rmat16_routes(hy, rmat16, algo, force):
    """R-MAT scale 16, budget 25 % of the edge bytes the algorithm reads."""
    e = engine(hy, rmat16, edge_bytes(rmat16, algo) // 4, force_route=force, seed=7)
    src = 0 if algo != "ppr" else 5
    got = e.run(algo, None if algo == "pagerank" else src)
    check(rmat16, algo, got, src)
    st = e.stats()
    assert st["edges_relaxed"] > 0
    if force in (2, 3, 4):
        others = [r for r in (1, 2, 3, 4) if r != force]
        assert st["route_partitions"][force] > 0
        assert all(st["route_partitions"][r] == 0 for r in others)
    e.close()


@pytest.mark.parametrize("force", FORCE)
def test_rmat16_cc(hy, rmat16_sym, force):
    e = engine(hy, rmat16_sym, edge_bytes(rmat16_sym, "cc") // 4, force_route=force, seed=3)
    check(rmat16_sym, "cc", e.run("cc"))
    e.close()


@pytest.mark.parametrize("algo", ["bfs", "sssp", "pagerank"])
def test_all_cached(hy, rmat16, algo):
    """A budget larger than the graph: every partition resident (cache route only)."""
    e = engine(hy, rmat16, 4 * edge_bytes(rmat16, algo), force_route=1)
    got = e.run(algo, None if algo == "pagerank" else 0)
    check(rmat16, algo, got)
    st = e.stats()
    assert st["route_partitions"][1] > 0
    assert sum(st["route_partitions"][2:]) == 0
    assert e.info()["n_cached"] == e.info()["n_parts"]
    e.close()


def test_all_four_routes_fire_under_cost_model(hy, rmat16):
    """With a small MR the cost model uses cache, F, C and Z across SSSP iterations."""
    e = engine(hy, rmat16, edge_bytes(rmat16, "sssp") // 4, MR=4)
    check(rmat16, "sssp", e.run("sssp", 0))
    rp = e.stats()["route_partitions"]
    assert all(rp[r] > 0 for r in (1, 2, 3, 4)), rp
    e.close()


IRREGULAR = [
    dict(V=1, E=0), dict(V=1, E=3), dict(V=33, E=100), dict(V=1000, E=1), dict(V=4097, E=30000),
    dict(V=5000, E=80000, skew=1.3), dict(V=12345, E=200000, skew=0.9),
]


@pytest.mark.parametrize("spec", IRREGULAR, ids=lambda s: f"V{s['V']}E{s['E']}")
@pytest.mark.parametrize("force", [-1, 2, 3, 4, 5])
def test_irregular_graphs(hy, spec, force):
    g = gg.random_graph(spec["V"], spec["E"], seed=spec["V"] + spec["E"], skew=spec.get("skew", 0.0))
    s = gg.symmetrize(g)
    budget = max(64 * 1024, g.E * 2)
    e = engine(hy, g, budget, force_route=force, part_bytes=4096, seed=11)
    srcs = sorted({0, g.V - 1, g.V // 2})
    for src in srcs:
        check(g, "bfs", e.run("bfs", src), src)
        check(g, "sssp", e.run("sssp", src), src)
    if g.V > 1:
        check(g, "pagerank", e.run("pagerank"))
    e.close()
    e = engine(hy, s, max(64 * 1024, s.E * 2), force_route=force, part_bytes=4096, seed=12)
    check(s, "cc", e.run("cc"))
    e.close()


def test_hub_larger_than_partition(hy):
    """A star whose centre alone exceeds the partition size (single-word partition)."""
    L = 50000
    off = np.zeros(L + 2, np.uint64)
    off[1:] = L
    off[-1] = L + 0
    dst = np.arange(1, L + 1, dtype=np.uint32)
    g = gg.CSR(L + 1, L, off, dst, np.full(L, 3, np.uint32))
    e = engine(hy, g, 8 * L * 4, part_bytes=4096)
    vb = e.partitions()
    assert vb[1] == 32  # the centre's word forms a partition with more than part_edges edges
    for force in (-1, 2, 3, 4):
        e.set_param("force_route", force)
        check(g, "bfs", e.run("bfs", 0))
        check(g, "sssp", e.run("sssp", 0))
    e.close()


def test_mesh_high_diameter(hy):
    g = gg.mesh(256, 128, shortcut_frac=0.001, radius=16, wmax=1000)
    e = engine(hy, g, g.E * 8 // 5, part_bytes=16384)   # 20 % of dst + weight bytes
    check(g, "bfs", e.run("bfs", 0))
    check(g, "sssp", e.run("sssp", 0))
    check(g, "cc", e.run("cc"))
    assert e.stats()["iterations"] > 20
    e.close()


def internal_graph(e, g):
    """The graph in the engine's internal (hub-sorted) vertex order, built by the oracle."""
    perm = e.permutation()
    assert perm.tolist() == pl.hub_order(g.off, g.dst, e.get_param("hub_frac"))
    off2, dst2, w2 = pl.relabel(g.off, g.dst, g.w, perm.tolist())
    return gg.CSR(g.V, g.E, off2, dst2, w2), perm


@pytest.mark.parametrize("hub_frac", [0.0, 0.08])
def test_partition_table_matches_oracle(hy, rmat16, hub_frac):
    for pb in (4096, 64 * 1024, 1 << 20, 4 << 20):
        e = engine(hy, rmat16, 1 << 24, part_bytes=pb, hub_frac=hub_frac)
        g2, _ = internal_graph(e, rmat16)
        assert e.partitions().tolist() == pl.partition_bounds(g2.off, pb // 4)
        e.close()


@pytest.mark.parametrize("algo", ["bfs", "sssp", "pagerank"])
def test_planner_matches_oracle(hy, rmat16, algo):
    """Cost analysis and engine selection on the device (Alg. 1) against the
    exact-rational oracle, on random frontiers of several densities
    (PageRank's planning walks the bitmap with the dense mapping)."""
    params = dict(alpha=0.8, beta=0.4, gamma=0.625, MR=8)
    e = engine(hy, rmat16, edge_bytes(rmat16, algo) // 4, **params)
    vb = e.partitions()
    g2, perm = internal_graph(e, rmat16)
    E_part = np.diff(g2.off[vb.astype(np.int64)].astype(np.int64))
    rng = np.random.default_rng(5)
    d1 = 8 if algo == "sssp" else 4
    n_arrays = 2 if algo == "sssp" else 1
    for dens in (1e-4, 1e-3, 0.01, 0.1, 0.5, 1.0):
        act = (rng.random(rmat16.V) < dens).astype(np.uint8)
        routes, counts = e.plan(algo, act)
        na, ae, ln = orc.partition_counts(g2, act[perm], vb, 4, n_arrays, 128)
        assert np.array_equal(counts[:, 0], na) and np.array_equal(counts[:, 1], ae)
        assert np.array_equal(counts[:, 2], ln)
        n_cached = e.info()["n_cached"]
        want = pl.plan(E_part, na, ae, ln, d1, resident=range(n_cached), m=128, MR=8,
                       alpha=Fraction("0.8"), beta=Fraction("0.4"), gamma=Fraction("0.625"))
        assert routes.tolist() == want, dens
    e.close()


@pytest.mark.parametrize("algo", ["bfs", "sssp", "cc", "pagerank"])
def test_without_hub_sorting(hy, rmat16, rmat16_sym, algo):
    g = rmat16_sym if algo == "cc" else rmat16
    e = engine(hy, g, edge_bytes(g, algo) // 4, hub_frac=0.0)
    assert e.permutation().tolist() == list(range(g.V))
    check(g, algo, e.run(algo, 0 if algo in ("bfs", "sssp") else None))
    e.close()


@pytest.mark.parametrize("delta", [0, 1, 7, 100, -1])
def test_sssp_delta_stepping(hy, rmat16, delta):
    """Bucketed SSSP (any bucket width, 0 = one bucket) reaches the same distances."""
    e = engine(hy, rmat16, edge_bytes(rmat16, "sssp") // 4, sssp_delta=delta)
    for src in (0, 17):
        check(rmat16, "sssp", e.run("sssp", src), src)
    e.close()


@pytest.mark.parametrize("delta", [0, 50, 1000, -1])
def test_mesh_sssp_buckets(hy, delta):
    g = gg.mesh(300, 200, shortcut_frac=0.001, radius=16, wmax=1000)
    e = engine(hy, g, g.E * 8 // 5, part_bytes=16384, sssp_delta=delta)
    check(g, "sssp", e.run("sssp", 0))
    e.close()


def test_cc_long_chain(hy):
    """A directed-both-ways path numbered in reverse: min-label propagation alone
    needs one iteration per vertex; pointer jumping must give the same labels."""
    n = 5000
    src = np.concatenate([np.arange(1, n), np.arange(0, n - 1)])
    dst = np.concatenate([np.arange(0, n - 1), np.arange(1, n)])
    order = np.lexsort((dst, src))
    off = np.concatenate([[0], np.cumsum(np.bincount(src, minlength=n))]).astype(np.uint64)
    g = gg.CSR(n, len(src), off, dst[order].astype(np.uint32), None)
    for hub in (0.0, 0.08):
        e = engine(hy, g, 1 << 20, part_bytes=4096, hub_frac=hub)
        check(g, "cc", e.run("cc"))
        assert e.stats()["iterations"] < n // 4
        e.close()


def test_budget_and_argument_errors(hy, rmat16):
    e = hy.Engine(params={"part_bytes": 64 * 1024})
    e.load(rmat16)
    with pytest.raises(hy.HytgError) as ex:
        e.set_budget(1024)
    assert ex.value.status == hy.HYTG_ERR_BUDGET
    with pytest.raises(hy.HytgError) as ex:
        e.run("bfs", 0)
    assert ex.value.status in (hy.HYTG_ERR_BUDGET, hy.HYTG_ERR_STATE)
    e.set_budget(1 << 22)
    with pytest.raises(hy.HytgError) as ex:
        e.run("bfs", rmat16.V)
    assert ex.value.status == hy.HYTG_ERR_ARG
    with pytest.raises(hy.HytgError) as ex:
        e.set_param("no_such_key", 1)
    assert ex.value.status == hy.HYTG_ERR_ARG
    check(rmat16, "bfs", e.run("bfs", 0))    # context still usable after errors
    e.close()
    g = gg.random_graph(100, 300, seed=1, weights=False)
    e = engine(hy, g, 1 << 20)
    with pytest.raises(hy.HytgError) as ex:
        e.run("sssp", 0)
    assert ex.value.status == hy.HYTG_ERR_ARG
    e.close()


def test_cc_needs_symmetric_csr(hy, rmat16, rmat16_sym):
    """CC is weakly connected components and needs a symmetric CSR: a directed
    graph, or one whose reverse edges differ in multiplicity, is refused with
    HYTG_ERR_ARG, and the context stays usable."""
    e = engine(hy, rmat16, edge_bytes(rmat16, "cc") // 4)
    with pytest.raises(hy.HytgError) as ex:
        e.run("cc")
    assert ex.value.status == hy.HYTG_ERR_ARG
    check(rmat16, "bfs", e.run("bfs", 0))
    e.load(rmat16_sym)
    check(rmat16_sym, "cc", e.run("cc"))
    e.close()
    g = gg.CSR(3, 4, np.array([0, 2, 3, 4], np.uint64), np.array([1, 1, 0, 2], np.uint32), None)
    e = engine(hy, g, 1 << 20)
    with pytest.raises(hy.HytgError) as ex:
        e.run("cc")
    assert ex.value.status == hy.HYTG_ERR_ARG
    check(g, "bfs", e.run("bfs", 0))
    e.close()


def test_hostmem_failure_injected(hy, rmat16, monkeypatch):
    """A pinned allocation that fails (made on the host by
    HYTG_INJECT_HOSTMEM_FAIL) gives HYTG_ERR_HOSTMEM and leaves the context
    usable: the next load and run succeed."""
    e = hy.Engine(params={"part_bytes": 64 * 1024})
    monkeypatch.setenv("HYTG_INJECT_HOSTMEM_FAIL", "1")
    with pytest.raises(hy.HytgError) as ex:
        e.load(rmat16)
    assert ex.value.status == hy.HYTG_ERR_HOSTMEM
    with pytest.raises(hy.HytgError) as ex:
        e.run("bfs", 0)
    assert ex.value.status == hy.HYTG_ERR_STATE
    monkeypatch.delenv("HYTG_INJECT_HOSTMEM_FAIL")
    e.load(rmat16)
    e.set_budget(edge_bytes(rmat16, "bfs") // 4)
    check(rmat16, "bfs", e.run("bfs", 0))
    e.close()


@pytest.mark.parametrize("algo", ["bfs", "sssp", "pagerank"])
def test_host_huge_pages(hy, rmat16, algo):
    """Edge arrays in transparent-huge-page memory registered with the driver
    ("host_huge" = 1, off by default) give the same results on every route."""
    e = hy.Engine(params={"part_bytes": 64 * 1024, "host_huge": 1})
    assert e.get_param("host_huge") == 1
    e.load(rmat16)
    e.set_budget(edge_bytes(rmat16, algo) // 4)
    check(rmat16, algo, e.run(algo, 0 if algo != "pagerank" else None))
    e.close()


@pytest.mark.parametrize("algo", ["bfs", "sssp", "pagerank"])
def test_staging_slot_reuse(hy, rmat16, algo):
    """F tasks that a staging slot still holds run without a copy; results
    are unchanged, and for BFS/SSSP (whose F sets per iteration do not
    depend on the order of the tasks) copied plus reused bytes equal the
    bytes copied with reuse off.  BFS/SSSP run on a mesh, whose frontier
    band stays in the same few partitions for many iterations."""
    if algo == "pagerank":
        g, pb = rmat16, 64 * 1024
    else:
        g, pb = gg.mesh(256, 128, shortcut_frac=0.0, wmax=1000), 16384
    runs = {}
    for reuse in (0, 1):
        e = engine(hy, g, edge_bytes(g, algo) // 4, part_bytes=pb, force_route=2, slot_reuse=reuse)
        assert e.get_param("slot_reuse") == reuse
        src = None if algo == "pagerank" else 0
        for _ in range(2):                     # the second run can reuse the first's slots
            check(g, algo, e.run(algo, src))
        runs[reuse] = e.stats()
        e.close()
    off, on = runs[0], runs[1]
    assert off["f_reused_tasks"] == 0 and off["f_reused_bytes"] == 0
    assert on["f_reused_tasks"] > 0
    if algo != "pagerank":
        assert on["link_bytes"][2] + on["f_reused_bytes"] == off["link_bytes"][2]
        assert on["f_tasks"] == off["f_tasks"]


@pytest.mark.parametrize("algo", ["bfs", "sssp", "pagerank"])
def test_copies_ahead(hy, rmat16, algo):
    """F tasks copied ahead at the end of an iteration ("f_ahead") for the
    next one give the same results; the next iterations run some tasks from
    those copies, and each copy ahead is counted in the F link bytes.  The
    engine is run twice, so the second run starts with the first one's
    slots and ring position, and once with the device loop off."""
    # one partition per task and a staging share that holds several slots (a
    # copy ahead needs a slot beyond the ones in use; on R-MAT 16 the first
    # 32 vertices, one partition, hold about 100 K edges)
    if algo == "pagerank":
        g, pb, budget, sf = rmat16, 64 * 1024, edge_bytes(rmat16, algo), 0.75
    else:
        g = gg.mesh(256, 128, shortcut_frac=0.0, wmax=1000)
        pb, budget, sf = 16384, edge_bytes(g, algo) // 2, 0.5
    src = None if algo == "pagerank" else 0
    base = engine(hy, g, budget, part_bytes=pb, force_route=2, k=1, staging_frac=sf)
    ref = base.run(algo, src)
    ref_st = base.stats()
    assert base.info()["n_slots"] >= 4
    base.close()
    for loop in (1, 0):
        e = engine(hy, g, budget, part_bytes=pb, force_route=2, k=1, staging_frac=sf, f_ahead=3,
                   device_loop=loop)
        assert e.get_param("f_ahead") == 3
        for _ in range(2):
            got = e.run(algo, src)
            check(g, algo, got)
            st = e.stats()
            assert st["f_ahead_tasks"] > 0 and st["f_ahead_hits"] > 0
            assert st["f_ahead_hits"] <= st["f_ahead_tasks"]
            if algo != "pagerank":
                assert np.array_equal(got, ref)
                # the same F sets per iteration (min-updates): tasks run from a
                # copy ahead are not copied again, and copies ahead count as F bytes
                assert st["f_tasks"] == ref_st["f_tasks"]
                missed = st["link_bytes"][2] - ref_st["link_bytes"][2]
                assert missed >= 0
        e.close()


@pytest.mark.parametrize("algo", ["bfs", "sssp", "pagerank", "cc"])
def test_copy_kernel(hy, rmat16, rmat16_sym, algo):
    """F copies by a kernel over mapped host memory ("f_copy" blocks per SM)
    in place of the copy engine give the same results, alone and with copies
    ahead.  The kernel starts at the 16-byte boundary at or below a task's
    first edge, so it reads at most 3 words more per array and task."""
    g = rmat16_sym if algo == "cc" else rmat16
    src = None if algo in ("pagerank", "cc") else 0
    narr = 2 if algo == "sssp" else 1
    runs = {}
    for fc, fa in ((0, 0), (2, 0), (1, 2)):
        e = engine(hy, g, edge_bytes(g, algo), force_route=2, k=1, staging_frac=0.75, f_copy=fc, f_ahead=fa)
        assert e.get_param("f_copy") == fc
        got = e.run(algo, src)
        check(g, algo, got)
        runs[(fc, fa)] = (got, e.stats())
        e.close()
    ref, st0 = runs[(0, 0)]
    got, st = runs[(2, 0)]
    if algo != "pagerank":
        assert np.array_equal(got, ref)
        assert st["f_tasks"] == st0["f_tasks"]
        extra = st["link_bytes"][2] - st0["link_bytes"][2]
        assert 0 <= extra <= 3 * 4 * narr * st["f_tasks"]
    assert st["kernel_launches"] > st0["kernel_launches"]


def test_sssp_overflow(hy):
    g = gg.CSR(4, 3, np.array([0, 1, 2, 3, 3], np.uint64), np.array([1, 2, 3], np.uint32),
               np.array([0x7FFFFFFF, 0x7FFFFFFF, 5], np.uint32))
    e = engine(hy, g, 1 << 20)
    with pytest.raises(hy.HytgError) as ex:
        e.run("sssp", 0)
    assert ex.value.status == hy.HYTG_ERR_OVERFLOW
    check(g, "bfs", e.run("bfs", 0))
    e.close()


def test_invalid_csr_rejected(hy):
    g = gg.random_graph(50, 100, seed=2)
    bad = gg.CSR(g.V, g.E, g.off.copy(), g.dst.copy(), g.w)
    bad.dst[3] = g.V
    e = hy.Engine()
    with pytest.raises(hy.HytgError) as ex:
        e.load(bad)
    assert ex.value.status == hy.HYTG_ERR_ARG
    e.close()


def test_pagerank_bound_reported(hy, rmat16):
    e = engine(hy, rmat16, edge_bytes(rmat16, "pagerank") // 4)
    got = e.run("pagerank")
    check(rmat16, "pagerank", got)
    st = e.stats()
    rank, delta = e.pagerank_state()
    B = st["pr_residual_sum"] / ((1 - 0.85) * st["pr_rank_sum"])
    assert B < 1e-4
    assert abs(float(rank.astype(np.float64).sum()) - st["pr_rank_sum"]) < 1e-3 * st["pr_rank_sum"]
    e.close()


def test_probes(hy):
    e = hy.Engine()
    mc, zc = e.probe_link(64 << 20, 2)
    assert mc > 1 and zc > 1
    uni, skew = e.probe_atomics(1 << 22, 2)
    assert uni > 1 and skew > 0.1
    for width in (1, 2, 4):
        assert hy.hytg_probe_frame_push(e.ctx, 1 << 20, 1, width) > 0.01
    with pytest.raises(hy.HytgError) as ex:
        hy.hytg_probe_frame_push(e.ctx, 1 << 20, 1, 3)
    assert ex.value.status == hy.HYTG_ERR_ARG
    e.close()


@pytest.mark.parametrize("algo", ["bfs", "sssp", "cc", "pagerank", "ppr"])
@pytest.mark.parametrize("force", [-1, 2, 5])
def test_two_pass(hy, rmat16, rmat16_sym, algo, force):
    """Second pass over resident partitions (Sec. VI-A) leaves results unchanged."""
    g = rmat16_sym if algo == "cc" else rmat16
    e = engine(hy, g, edge_bytes(g, algo) // 4, two_pass=2, force_route=force, seed=3,
               two_pass_min_degree=0)
    src = {"bfs": 0, "sssp": 0, "ppr": 5}.get(algo)
    check(g, algo, e.run(algo, src), 0 if src is None else src)
    if force == 2 and algo != "ppr":
        assert e.stats()["extra_edges"] > 0
    # ranges below the minimum mean degree get no second pass; results stay
    e.set_param("two_pass_min_degree", 1e6)
    check(g, algo, e.run(algo, src), 0 if src is None else src)
    if force == 2:
        assert e.stats()["extra_edges"] == 0
    e.close()


def test_two_pass_mesh_buckets(hy):
    g = gg.mesh(300, 200, shortcut_frac=0.001, radius=16, wmax=1000)
    e = engine(hy, g, g.E * 8 // 5, part_bytes=16384, two_pass=2)
    check(g, "sssp", e.run("sssp", 0))
    check(g, "bfs", e.run("bfs", 0))
    check(g, "cc", e.run("cc"))
    e.close()


@pytest.mark.parametrize("algo", ["pagerank", "ppr"])
@pytest.mark.parametrize("prio", [0, 1])
@pytest.mark.parametrize("force", [-1, 2])
def test_delta_first_order(hy, rmat16, algo, prio, force):
    """F tasks in delta-first order (Sec. VI-A) or partition order: the same
    fixed point within the PageRank tolerance."""
    e = engine(hy, rmat16, edge_bytes(rmat16, algo) // 4, priority=prio, force_route=force)
    src = 5 if algo == "ppr" else None
    check(rmat16, algo, e.run(algo, src), 5 if src is not None else 0)
    assert e.stats()["f_tasks"] > 0
    e.close()


@pytest.mark.parametrize("k", [1, 2, 4])
def test_task_combination_matches_planner(hy, rmat16_sym, k):
    """Alg. 1's task combination (Sec. V-B) as the engine issues it: the F
    copies of CC's first iteration (every vertex active), read from the launch
    timeline, are exactly the oracle planner's groups of the same routes (at
    most k consecutive F partitions within a staging slot's capacity)."""
    g = rmat16_sym
    e = engine(hy, g, edge_bytes(g, "cc") // 4, k=k, device_loop=0, timing=1)
    routes, _ = e.plan("cc", np.ones(g.V, np.uint8))
    vb = e.partitions()
    deg = np.diff(g.off.astype(np.int64))[e.permutation()]      # internal vertex order
    off_int = np.concatenate([[0], np.cumsum(deg)])
    E_part = off_int[vb[1:]] - off_int[vb[:-1]]
    groups, _, _, _ = pl.combine_tasks([int(r) for r in routes], k=k, E_part=E_part,
                                       cap_edges=e.info()["slot_edges"])
    assert len(groups) > 1
    check(g, "cc", e.run("cc"))
    tl = e.timeline()
    bins = np.flatnonzero(tl["kind"] == 2)
    first = tl[bins[0]:bins[1]] if len(bins) > 1 else tl[bins[0]:]
    copies = first[first["kind"] == 8]
    got = [list(range(int(r["part_first"]), int(r["part_last"]) + 1)) for r in copies]
    assert got == groups
    relaxes = first[first["kind"] == 4]
    assert [(int(r["part_first"]), int(r["part_last"])) for r in relaxes] == [(x[0], x[-1]) for x in groups]
    e.close()
