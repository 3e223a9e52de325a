"""Batched runs: many BFS/SSSP sources or PPR seeds in one run that shares
every partition transfer.  Each source's row must equal the single-source
oracle result (BFS/SSSP bit-exact, PPR within 1e-4 L1 of the normalised
vector), for every route and with hub sorting on or off."""
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
def rmat16():
    return gg.rmat(16, seed=1)


def sources_with_out_edges(g, n, seed):
    """Seeded draws among vertices with at least one out-edge (vertex 0 first,
    one duplicate), as the batched workload specifies."""
    rng = np.random.default_rng(seed)
    cand = np.flatnonzero(np.diff(g.off.astype(np.int64)) > 0)
    src = [0] + rng.choice(cand, n - 2, replace=False).tolist()
    src.append(src[1])
    return src


def engine(hy, g, budget, **params):
    e = hy.Engine(params={"part_bytes": 64 * 1024, **params})
    e.load(g)
    e.set_budget(int(budget))
    return e


@pytest.mark.parametrize("force", [-1, 2, 3, 4, 5])
def test_batched_bfs_64(hy, rmat16, force):
    g = rmat16
    src = sources_with_out_edges(g, 64, 1)
    e = engine(hy, g, g.E, force_route=force, seed=5)
    got = e.run("bfs", src)
    assert got.shape == (64, g.V)
    for s, v in enumerate(src):
        want, _ = orc.bfs(g, v)
        assert np.array_equal(got[s], want), f"source {s} ({v})"
    st = e.stats()
    assert st["n_sources"] == 64
    plain = sum(orc.bfs(g, v)[1] for v in src)
    assert st["source_edges"] == plain       # each source relaxes each reached edge once
    e.close()


@pytest.mark.parametrize("force,hub", [(-1, 0.08), (4, 0.0), (2, 0.08), (3, 0.08)])
def test_batched_sssp_64(hy, rmat16, force, hub):
    g = rmat16
    src = sources_with_out_edges(g, 64, 2)
    e = engine(hy, g, g.E * 2, force_route=force, hub_frac=hub)
    got = e.run("sssp", src)
    for s, v in enumerate(src):
        want, _, _ = orc.sssp(g, v)
        assert np.array_equal(got[s], want), f"source {s} ({v})"
    e.close()


@pytest.mark.parametrize("sparse_below", [0, 65])
def test_batched_sssp_relax_forms(hy, rmat16, sparse_below):
    """Both forms of the batched SSSP relax (a lane per source, a lane per
    edge looping over its sources) give every source's exact distances."""
    g = rmat16
    src = sources_with_out_edges(g, 40, 6)
    e = engine(hy, g, g.E * 2, batch_sparse_below=sparse_below)
    got = e.run("sssp", src)
    for s, v in enumerate(src):
        assert np.array_equal(got[s], orc.sssp(g, v)[0]), f"source {s} ({v})"
    e.close()


def test_batched_sssp_matches_plain_small_k(hy, rmat16):
    g = rmat16
    src = sources_with_out_edges(g, 5, 3)
    e = engine(hy, g, g.E * 2)
    got = e.run("sssp", src)
    for s, v in enumerate(src):
        assert np.array_equal(got[s], e.run("sssp", v))
    e.close()


@pytest.mark.parametrize("force,K", [(-1, 32), (4, 32), (2, 32), (3, 32), (2, 13), (-1, 5)])
def test_batched_ppr(hy, rmat16, force, K):
    """Every route (F with the batched second pass), full and partial frames
    of 8 seeds: the vector push adds whole frames, so seeds that are not
    taken, or do not exist, must carry zero messages."""
    g = rmat16
    src = sources_with_out_edges(g, K, 4)
    e = engine(hy, g, g.E, force_route=force)
    got = e.run("ppr", src)
    assert got.shape == (K, g.V)
    for s, v in enumerate(src):
        x, _, _ = orc.pagerank(g, tol=1e-13, seed=v)
        err = float(np.abs(got[s].astype(np.float64) - x).sum())
        assert err <= 1e-4, f"seed {s} ({v}): L1 {err}"
    e.close()


def test_batched_irregular(hy):
    g = gg.random_graph(1000, 6000, seed=12, skew=1.2)
    src = [0, 999, 500, 500, 3, 17, 64, 65]
    e = engine(hy, g, 1 << 20, part_bytes=4096)
    lv = e.run("bfs", src)
    d = e.run("sssp", src)
    for s, v in enumerate(src):
        assert np.array_equal(lv[s], orc.bfs(g, v)[0])
        assert np.array_equal(d[s], orc.sssp(g, v)[0])
    e.close()


def test_batched_limits(hy, rmat16):
    e = engine(hy, rmat16, rmat16.E)
    with pytest.raises(hy.HytgError) as ex:
        e.run("bfs", list(range(65)))
    assert ex.value.status == hy.HYTG_ERR_ARG
    with pytest.raises(hy.HytgError) as ex:
        e.run("ppr", list(range(33)))
    assert ex.value.status == hy.HYTG_ERR_ARG
    # a single-source run after a batched one uses the plain path again
    assert np.array_equal(e.run("bfs", 0), orc.bfs(rmat16, 0)[0])
    e.close()


def test_autotune_keeps_results(hy, rmat16):
    from paper_2208_14935_gb300.autotune import autotune
    g = rmat16
    e = engine(hy, g, g.E)
    space = {"part_bytes": [32 * 1024, 128 * 1024], "k": [2, 8], "MR": [16, 256]}
    best = autotune(e, [("bfs", [0]), ("sssp", [0])], space=space, reps=1)
    assert set(best) == set(space)
    for k, v in best.items():
        assert e.get_param(k) == v
    assert np.array_equal(e.run("bfs", 0), orc.bfs(g, 0)[0])
    assert np.array_equal(e.run("sssp", 0), orc.sssp(g, 0)[0])
    e.close()
