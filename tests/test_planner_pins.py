"""Pins the cost-model oracle (Sec. V) to hand-computed values (no GPU)."""
import json
import os
from fractions import Fraction

import numpy as np

from gen import graphgen as gg
from oracle import oracle as orc
from oracle import planner as pl

NAMES = {"Z": pl.ROUTE_Z, "F": pl.ROUTE_F, "C": pl.ROUTE_C, "-": pl.ROUTE_NONE}


def test_cost_model_hand_cases(golden_dir):
    fx = json.load(open(os.path.join(golden_dir, "cost_model_hand.json")))
    for c in fx["cases"]:
        Tef, Tec, Tiz = pl.costs(c["E_i"], c["act_edges"], c["n_act"], c["lines"], c["d1"])
        assert (Tef, Tec, Tiz) == (Fraction(c["Tef"]), Fraction(c["Tec"]), Fraction(c["Tiz"])), c["name"]
        assert pl.select_route(Tef, Tec, Tiz) == NAMES[c["route"]], c["name"]


def test_cost_invariants():
    # Sec. III-C / Fig. 4: equal active edges, more active vertices -> more requests -> Tiz no lower
    E_i = 1 << 20
    for nv_small, nv_big in [(3, 6), (10, 100), (100, 5000)]:
        a = pl.costs(E_i, 64 * 100, nv_small, nv_small, 4, MR=1)[2]
        b = pl.costs(E_i, 64 * 100, nv_big, nv_big, 4, MR=1)[2]
        assert b > a
    # every edge of the partition active: Tec = Tef + index term >= Tef, so never C (alpha < 1)
    for E_i in (1000, 32768, 1 << 20, 12345679):
        for nv in (1, 17, 1000):
            Tef, Tec, Tiz = pl.costs(E_i, E_i, nv, nv, 4)
            assert Tec >= Tef
            assert pl.select_route(Tef, Tec, Tiz) != pl.ROUTE_C
    # an aligned 32-edge list of 4-byte entries is one line; shifted by one entry, two lines
    off = np.array([0, 32, 64, 97, 97], np.uint64)
    g = gg.CSR(4, 97, off, np.zeros(97, np.uint32), None)
    act = np.array([1, 0, 0, 1], np.uint8)
    na, ae, ln = orc.partition_counts(g, act, [0, 4])
    assert (na[0], ae[0], ln[0]) == (2, 32, 1)      # vertex 3 has degree 0 -> 0 lines
    off2 = np.array([0, 1, 33, 33], np.uint64)
    g2 = gg.CSR(3, 33, off2, np.zeros(33, np.uint32), None)
    na, ae, ln = orc.partition_counts(g2, np.array([0, 1, 0], np.uint8), [0, 3])
    assert (na[0], ae[0], ln[0]) == (1, 32, 2)
    na, ae, ln = orc.partition_counts(g2, np.array([0, 1, 0], np.uint8), [0, 3], n_arrays=2)
    assert ln[0] == 4


def test_counts_brute_force_random():
    rng = np.random.default_rng(7)
    g = gg.random_graph(2000, 30000, seed=7, skew=1.1)
    vb = pl.partition_bounds(g.off, 2000)
    for _ in range(5):
        act = (rng.random(g.V) < rng.random()).astype(np.uint8)
        na, ae, ln = orc.partition_counts(g, act, vb)
        for i in range(len(vb) - 1):
            vs = [v for v in range(vb[i], vb[i + 1]) if act[v]]
            assert na[i] == len(vs)
            assert ae[i] == sum(int(g.off[v + 1] - g.off[v]) for v in vs)
            L = 0
            for v in vs:
                lines = {b // 128 for b in range(4 * int(g.off[v]), 4 * int(g.off[v + 1]))}
                L += len(lines)
            assert ln[i] == L


def test_partition_bounds_hand(golden_dir):
    fx = json.load(open(os.path.join(golden_dir, "partition_and_combine_hand.json")))["partition"]
    deg = np.zeros(fx["V"], np.uint64)
    for v, d in fx["degree_by_vertex"].items():
        deg[int(v)] = d
    off = np.concatenate([[0], np.cumsum(deg)]).astype(np.uint64)
    assert pl.partition_bounds(off, fx["part_edges"]) == fx["bounds"]


def test_partition_bounds_properties():
    for seed in range(5):
        g = gg.random_graph(5000 + 37 * seed, 60000, seed=seed, skew=1.3)
        pe = 1500 + 100 * seed
        b = pl.partition_bounds(g.off, pe)
        assert b[0] == 0 and b[-1] == g.V
        for lo, hi in zip(b[:-1], b[1:]):
            assert hi > lo
            assert lo % 32 == 0
            assert hi % 32 == 0 or hi == g.V
            ne = int(g.off[hi] - g.off[lo])
            assert ne <= pe or hi - lo <= 32           # over-full only for a single word
            if hi < g.V:                               # maximal: one more word would overflow
                nxt = min(hi + 32, g.V)
                assert int(g.off[nxt] - g.off[lo]) > pe


def test_task_combination_hand(golden_dir):
    fx = json.load(open(os.path.join(golden_dir, "partition_and_combine_hand.json")))["combine"]
    routes = [NAMES[r] for r in fx["routes"]]
    groups, vc, vz, vcache = pl.combine_tasks(routes, k=fx["k"])
    assert groups == fx["groups"] and vc == fx["vc"] and vz == fx["vz"] and vcache == []
    # every F partition appears in exactly one group (the printed loop would drop some)
    flat = [i for grp in groups for i in grp]
    assert flat == [i for i, r in enumerate(routes) if r == pl.ROUTE_F]


def test_task_combination_capacity():
    routes = [pl.ROUTE_F] * 6
    E = [10, 10, 25, 10, 10, 10]
    groups, _, _, _ = pl.combine_tasks(routes, k=4, E_part=E, cap_edges=30)
    assert groups == [[0, 1], [2], [3, 4, 5]]


def test_plan_resident_and_inactive():
    routes = pl.plan([100, 100, 100], [0, 2, 1], [0, 10, 0], [0, 2, 0], 4, resident=[0, 1])
    assert routes == [pl.ROUTE_NONE, pl.ROUTE_CACHE, pl.ROUTE_NONE]
