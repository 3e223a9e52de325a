"""Hub sorting (Sec. VI-A): the library's host ordering against the oracle's
restatement and a hand-worked case (no GPU needed: hytg_hub_order is host code)."""
import json
import os

import numpy as np
import pytest

from gen import graphgen as gg
from oracle import planner as pl


def _csr(V, edges):
    src = np.array([a for a, b in edges], np.int64)
    dst = np.array([b for a, b in edges], np.int64)
    order = np.lexsort((dst, src))
    off = np.concatenate([[0], np.cumsum(np.bincount(src, minlength=V))]).astype(np.uint64)
    return gg.CSR(V, len(edges), off, dst[order].astype(np.uint32), None)


@pytest.fixture(scope="module")
def hy():
    from paper_2208_14935_gb300 import build, hytg
    build.build()
    return hytg


def test_hub_order_hand(hy, golden_dir):
    fx = json.load(open(os.path.join(golden_dir, "hub_sort_hand.json")))
    g = _csr(fx["V"], fx["edges"])
    want = pl.hub_order(g.off, g.dst, fx["frac"])
    assert want[:2] == fx["perm_head"]
    assert want[2:] == [v for v in range(fx["V"]) if v not in fx["perm_head"]]
    perm, nh = hy.hytg_hub_order(g, fx["frac"])
    assert nh == 2 and perm.tolist() == want


@pytest.mark.parametrize("seed,frac", [(1, 0.08), (2, 0.3), (3, 0.0), (4, 1.0), (5, 0.08)])
def test_hub_order_matches_oracle(hy, seed, frac):
    g = gg.random_graph(3000 + seed, 20000, seed=seed, skew=1.2)
    perm, nh = hy.hytg_hub_order(g, frac)
    assert nh == int(frac * g.V)
    assert perm.tolist() == pl.hub_order(g.off, g.dst, frac)
    assert sorted(perm.tolist()) == list(range(g.V))


def test_hub_order_rmat(hy):
    g = gg.rmat(14, seed=1)
    perm, nh = hy.hytg_hub_order(g, 0.08)
    assert perm.tolist() == pl.hub_order(g.off, g.dst, 0.08)
    # hubs first: D_o * D_i is non-increasing over the first nh internal ids
    d_in = np.bincount(g.dst, minlength=g.V).astype(np.int64)
    h = np.diff(g.off.astype(np.int64)) * d_in
    assert np.all(np.diff(h[perm[:nh].astype(np.int64)]) <= 0)


def test_relabel_preserves_graph():
    g = gg.random_graph(500, 3000, seed=9, skew=1.0)
    perm = pl.hub_order(g.off, g.dst, 0.1)
    off2, dst2, w2 = pl.relabel(g.off, g.dst, g.w, perm)
    inv = np.empty(g.V, np.int64)
    inv[np.asarray(perm)] = np.arange(g.V)
    e1 = sorted((int(inv[u]), int(inv[v]), int(w)) for u in range(g.V)
                for v, w in zip(g.dst[g.off[u]:g.off[u + 1]], g.w[g.off[u]:g.off[u + 1]]))
    e2 = sorted((n, int(v), int(w)) for n in range(g.V)
                for v, w in zip(dst2[off2[n]:off2[n + 1]], w2[off2[n]:off2[n + 1]]))
    assert e1 == e2
