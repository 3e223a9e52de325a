"""Pins the CPU oracle to things other than itself (runs without a GPU).

Each algorithm is checked against brute force on tiny graphs, against an
alternate algorithm, against closed forms, and through O(E) certificates;
each certificate is shown to reject a planted mistake.
"""
import json
import os

import numpy as np
import pytest

from gen import graphgen as gg
from oracle import oracle as orc

UNR = orc.UNREACHED


def tiny_graphs(n_graphs=60, max_v=7, seed0=100):
    rng = np.random.default_rng(seed0)
    for t in range(n_graphs):
        V = int(rng.integers(1, max_v + 1))
        E = int(rng.integers(0, 3 * V + 1))
        yield gg.random_graph(V, E, seed=seed0 + t, wmax=9)


def brute_paths(g, src):
    """Minimum hop count and minimum weight over all simple directed paths."""
    V = g.V
    adj = [[] for _ in range(V)]
    for u in range(V):
        for e in range(int(g.off[u]), int(g.off[u + 1])):
            adj[u].append((int(g.dst[e]), int(g.w[e])))
    hops = [None] * V
    dist = [None] * V

    def dfs(u, seen, h, d):
        if hops[u] is None or h < hops[u]:
            hops[u] = h
        if dist[u] is None or d < dist[u]:
            dist[u] = d
        for v, w in adj[u]:
            if v not in seen:
                dfs(v, seen | {v}, h + 1, d + w)

    dfs(src, {src}, 0, 0)
    return ([UNR if x is None else x for x in hops], [UNR if x is None else x for x in dist])


def test_bfs_sssp_brute_force_tiny():
    n = 0
    for g in tiny_graphs():
        for src in range(g.V):
            hops, dist = brute_paths(g, src)
            lv, _ = orc.bfs(g, src)
            dd, _, ovf = orc.sssp(g, src)
            assert not ovf
            assert lv.tolist() == hops
            assert dd.tolist() == dist
            assert orc.sssp_bellman_ford(g, src).tolist() == dist
            assert orc.sssp_bellman_ford(g, src, unit_weights=True).tolist() == hops
            n += 1
    assert n > 100


def closure_labels(g):
    """Smallest id reachable in the undirected closure (boolean Floyd-Warshall)."""
    V = g.V
    R = np.eye(V, dtype=bool)
    for u in range(V):
        for e in range(int(g.off[u]), int(g.off[u + 1])):
            R[u, g.dst[e]] = R[g.dst[e], u] = True
    for k in range(V):
        R = R | (R[:, [k]] & R[[k], :])
    return [int(np.flatnonzero(R[v])[0]) for v in range(V)]


def test_cc_brute_force_tiny():
    for g in tiny_graphs(seed0=300):
        want = closure_labels(g)
        assert orc.cc(g).tolist() == want
        s = gg.symmetrize(g)
        assert orc.is_symmetric(s)
        assert orc.cc(s).tolist() == want
        assert orc.cc_bfs(s).tolist() == want


def csr_from_edges(V, edges):
    """CSR that keeps each row's edges in the given order (rows need not be sorted)."""
    rows = [[] for _ in range(V)]
    for u, v in edges:
        rows[u].append(v)
    off = np.zeros(V + 1, np.uint64)
    off[1:] = np.cumsum([len(r) for r in rows])
    dst = np.array([v for r in rows for v in r], dtype=np.uint32)
    return gg.CSR(V, len(dst), off, dst, None, "hand")


def brute_symmetric(g):
    """The definition: the multiset of edges (u, v) equals the multiset of (v, u)."""
    from collections import Counter
    pairs = Counter((u, int(g.dst[e])) for u in range(g.V) for e in range(int(g.off[u]), int(g.off[u + 1])))
    return all(pairs[(v, u)] == n for (u, v), n in pairs.items())


# (V, edges, symmetric): each False case defeats one plausible shortcut; a
# self-loop is its own reverse, so a graph of self-loops alone is symmetric.
SYMMETRY_CASES = [
    (3, [(0, 1), (1, 0), (1, 2)], False),                   # one reverse edge missing
    (2, [(0, 1), (0, 1), (1, 0)], False),                   # unequal multiplicity
    (3, [(0, 1), (1, 2), (2, 0)], False),                   # directed cycle: in-degree = out-degree everywhere
    (4, [(0, 1), (1, 0), (2, 3), (3, 3), (3, 2), (2, 2)], True),
    (3, [(0, 0), (2, 2), (2, 2)], True),                    # self-loops only
    (3, [(1, 1), (1, 2)], False),                           # self-loop beside a missing reverse
    (4, [(0, 3), (0, 1), (1, 0), (3, 0)], True),            # unsorted row, symmetric
    (4, [(0, 3), (0, 1), (1, 0), (3, 1), (1, 3), (3, 0), (2, 1)], False),
    (1, [], True),
]


@pytest.mark.parametrize("V,edges,want", SYMMETRY_CASES)
def test_is_symmetric_hand_cases(V, edges, want):
    g = csr_from_edges(V, edges)
    assert brute_symmetric(g) == want
    assert orc.is_symmetric(g) == want


def test_is_symmetric_brute_force_tiny():
    n_false = 0
    for g in tiny_graphs(seed0=400):
        want = brute_symmetric(g)
        assert orc.is_symmetric(g) == want
        n_false += not want
        assert orc.is_symmetric(gg.symmetrize(g))
    assert n_false > 20


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_alternates_agree_medium(seed):
    g = gg.random_graph(3000, 12000, seed=seed, skew=1.2, wmax=64)
    for src in (0, 7, 2999):
        lv, _ = orc.bfs(g, src)
        assert np.array_equal(lv, orc.sssp_bellman_ford(g, src, unit_weights=True))
        dd, _, _ = orc.sssp(g, src)
        assert np.array_equal(dd, orc.sssp_bellman_ford(g, src))
        assert orc.bfs_certify(g, src, lv)[0] == 0
        assert orc.sssp_certify(g, src, dd)[0] == 0
    s = gg.symmetrize(g)
    lab = orc.cc(s)
    assert np.array_equal(lab, orc.cc_bfs(s))
    assert orc.cc_certify(s, lab, len(np.unique(lab)))[0] == 0


def test_certificates_reject_planted_mistakes():
    g = gg.random_graph(500, 3000, seed=9, skew=1.0)
    lv, _ = orc.bfs(g, 0)
    reached = np.flatnonzero((lv != UNR) & (lv > 0))
    assert len(reached) > 10
    for v in reached[:5]:
        for delta in (-1, 1):
            bad = lv.copy()
            bad[v] = int(bad[v]) + delta
            assert orc.bfs_certify(g, 0, bad)[0] != 0
    bad = lv.copy()
    bad[reached[0]] = UNR
    assert orc.bfs_certify(g, 0, bad)[0] != 0

    dd, _, _ = orc.sssp(g, 0)
    for v in np.flatnonzero((dd != UNR) & (dd > 0))[:5]:
        for delta in (-1, 1):
            bad = dd.copy()
            bad[v] = int(bad[v]) + delta
            assert orc.sssp_certify(g, 0, bad)[0] != 0

    s = gg.symmetrize(g)
    lab = orc.cc(s)
    ncomp = len(np.unique(lab))
    big = np.flatnonzero(lab != np.arange(s.V))
    bad = lab.copy()
    bad[big[0]] = big[0]          # split a vertex off its component
    assert orc.cc_certify(s, bad, ncomp)[0] != 0
    bad = lab.copy()
    roots = np.unique(lab)
    bad[bad == roots[-1]] = roots[-2] if roots[-2] < roots[-1] else roots[-1]  # merge two
    if not np.array_equal(bad, lab):
        assert orc.cc_certify(s, bad, ncomp)[0] != 0


def test_sssp_overflow_flag():
    # a path of 3 edges with weights near 2^31 overflows the 32-bit result
    g = gg.CSR(4, 3, np.array([0, 1, 2, 3, 3], np.uint64), np.array([1, 2, 3], np.uint32),
               np.array([0x7FFFFFFF, 0x7FFFFFFF, 5], np.uint32))
    dd, _, ovf = orc.sssp(g, 0)
    assert ovf
    assert dd[1] == 0x7FFFFFFF and dd[3] == UNR


def dense_pagerank(g, d=0.85, seed=None):
    V = g.V
    M = np.zeros((V, V))
    deg = np.diff(g.off.astype(np.int64))
    for u in range(V):
        for e in range(int(g.off[u]), int(g.off[u + 1])):
            M[g.dst[e], u] += 1.0 / deg[u]
    t = np.ones(V) if seed is None else np.eye(V)[seed]
    x = np.linalg.solve(np.eye(V) - d * M, (1 - d) * t)
    return x


@pytest.mark.parametrize("seed", range(6))
def test_pagerank_against_dense_solve(seed):
    g = gg.random_graph(40 + seed, 160, seed=seed, skew=0.8)
    x, raw, it = orc.pagerank(g, tol=1e-15)
    xd = dense_pagerank(g)
    assert abs(raw - xd.sum()) < 1e-9 * xd.sum()
    assert np.abs(x - xd / xd.sum()).sum() < 1e-10
    xp, _, _ = orc.pagerank(g, tol=1e-15, seed=3)
    xpd = dense_pagerank(g, seed=3)
    assert np.abs(xp - xpd / xpd.sum()).sum() < 1e-10


def test_pagerank_closed_forms():
    d = 0.85
    n = 17   # directed cycle: every vertex has rank 1 (raw), 1/n normalised
    g = gg.CSR(n, n, np.arange(n + 1, dtype=np.uint64), ((np.arange(n) + 1) % n).astype(np.uint32), None)
    x, raw, _ = orc.pagerank(g, tol=1e-15)
    assert abs(raw - n) < 1e-9 and np.allclose(x, 1.0 / n, atol=1e-12)
    # star: centre 0 -> leaves 1..L, every leaf -> centre.
    L = 6
    off = np.array([0, L] + [L + i for i in range(1, L + 1)], np.uint64)
    dst = np.array(list(range(1, L + 1)) + [0] * L, np.uint32)
    g = gg.CSR(L + 1, 2 * L, off, dst, None)
    x, raw, _ = orc.pagerank(g, tol=1e-15)
    xc = (1 + d * L) / (1 + d)                 # x_c = (1-d) + d L x_l, x_l = (1-d) + d x_c / L
    xl = (1 - d) + d * xc / L
    assert abs(raw - (xc + L * xl)) < 1e-9
    assert abs(x[0] - xc / raw) < 1e-12 and np.allclose(x[1:], xl / raw, atol=1e-12)
    # no dangling vertex -> the raw fixed point sums to V exactly
    V = 50
    r = gg.random_graph(V, 200, seed=5)
    src = np.concatenate([np.repeat(np.arange(V), np.diff(r.off.astype(np.int64))), np.arange(V)])
    dst = np.concatenate([r.dst.astype(np.int64), (np.arange(V) + 1) % V])
    order = np.lexsort((dst, src))
    off = np.concatenate([[0], np.cumsum(np.bincount(src, minlength=V))]).astype(np.uint64)
    g = gg.CSR(V, len(dst), off, dst[order].astype(np.uint32), None)
    assert np.all(np.diff(g.off.astype(np.int64)) > 0)
    _, raw, _ = orc.pagerank(g, tol=1e-15)
    assert abs(raw - V) < 1e-8
    # with dangling vertices the mass leaks: raw sum strictly below V
    r2 = gg.random_graph(V, 200, seed=5, skew=1.0)
    _, raw2, _ = orc.pagerank(r2, tol=1e-15)
    assert np.any(np.diff(r2.off.astype(np.int64)) == 0) and raw2 < V - 1e-3


def test_pagerank_residual_bound():
    g = gg.random_graph(400, 2400, seed=4, skew=1.0)
    x, raw, _ = orc.pagerank(g, tol=1e-15)
    assert orc.pagerank_residual(g, x * raw) < 1e-9
    pert = x * raw
    pert[3] += 0.01
    res = orc.pagerank_residual(g, pert)
    # ||r - x*||_1 <= res / (1 - d)
    assert 0.01 <= res / 0.15 + 1e-12


def test_fig4_toy_graph_requests(golden_dir):
    fx = json.load(open(os.path.join(golden_dir, "fig4_toy_graph.json")))
    degs = fx["subset_green"]["degrees"] + fx["subset_grey"]["degrees"]
    assert len(degs) == fx["V"] and sum(degs) == fx["E"]
    for key in ("subset_green", "subset_grey"):
        sub = fx[key]
        assert sum(sub["degrees"]) == 64
        req = sum(-(-d * fx["entry_bytes"] // fx["m"]) for d in sub["degrees"])
        assert req == sub["requests"]
