"""ORACLE -- test infrastructure only.  Cost-aware task generation written out
from Sec. V of the paper in exact rational arithmetic (fractions.Fraction).

  partition_bounds  Sec. IV: edge-balanced chunk partitioning of the vertex
                    range into runs of consecutive vertices.
  costs             Sec. V-A, Eq. 1 (Tef), Eq. 2 (Tec, transfer term only as
                    the paper computes it in practice) and Eq. 3 (Tiz, with
                    RTT_zc = gamma RTT + (1 - gamma) (active/total edges) RTT).
  select_route      Sec. V-A engine selection (Alg. 1, cost analysis part).
  combine_tasks     Sec. V-B task combination (Alg. 1, combination part).

RTT is set to 1: it multiplies every cost and cancels in each comparison
(Sec. V-A, last sentence of "Transfer engine selection").

Readings where the text is silent or garbled (each also listed in the design
notes of the repository):
  * Partition boundaries fall on multiples of 32 vertices (one frontier
    bitmap word).  A partition is the longest such run whose edge count does
    not exceed `part_edges`; a single 32-vertex run with more edges forms a
    partition on its own.
  * d1 is the bytes read per edge, summed over the edge arrays the algorithm
    reads (4 for dst only, 8 for dst + weight); d2 = 8 (uint64 row offsets).
  * The line count of Eq. 3 is the exact number of m-byte lines spanned by
    each active vertex's segment of each edge array (footnote to Eq. 3).
  * Partitions with no active edges get no route.  A resident (cached)
    partition with active edges always takes the cache route, which has no
    transfer cost.
  * Comparisons are strict as printed: Tec == alpha Tef is not C; Tef == Tiz
    is ZC.
  * Alg. 1's combination loop, when an F partition meets a full group,
    closes the group and starts the next one with that partition (the
    printed loop would drop it).  Any non-F partition closes the open group.
    A group also closes before it would exceed the staging capacity.
"""
from __future__ import annotations

from fractions import Fraction
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np

ROUTE_NONE, ROUTE_CACHE, ROUTE_F, ROUTE_C, ROUTE_Z = 0, 1, 2, 3, 4

# Constants given in Sec. V: alpha = 80 %, beta = 40 %, gamma = 0.625 (after
# EMOGI), m = 128-byte requests, MR = 256 outstanding requests (PCIe 3.0),
# k = 4 partitions merged per F task, 32 MB partitions.
PAPER_ALPHA = Fraction(4, 5)
PAPER_BETA = Fraction(2, 5)
PAPER_GAMMA = Fraction(5, 8)
PAPER_M = 128
PAPER_MR = 256
PAPER_K = 4
PAPER_PART_BYTES = 32 * 1024 * 1024


def partition_bounds(off: np.ndarray, part_edges: int, align: int = 32) -> List[int]:
    """Vertex bounds [b_0 = 0, b_1, ..., b_N = V] of the chunk partitions."""
    V = len(off) - 1
    bounds = [0]
    b = 0
    while b < V:
        # largest aligned end e > b with off[e] - off[b] <= part_edges
        end = b
        nxt = min(b + align, V)
        while True:
            if int(off[nxt]) - int(off[b]) > part_edges:
                break
            end = nxt
            if nxt == V:
                break
            nxt = min(nxt + align, V)
        if end == b:
            end = min(b + align, V)
        bounds.append(end)
        b = end
    if V == 0:
        bounds.append(0)
    return bounds


def costs(E_i: int, act_edges: int, n_act: int, lines: int, d1: int, d2: int = 8,
          m: int = PAPER_M, MR: int = PAPER_MR, gamma: Fraction = PAPER_GAMMA
          ) -> Tuple[Fraction, Fraction, Fraction]:
    """(Tef_i, Tec_i, Tiz_i) of Eq. 1-3 with RTT = 1, as exact rationals."""
    def ceil_frac(x: Fraction) -> int:
        return -((-x.numerator) // x.denominator)

    Tef = Fraction(ceil_frac(Fraction(E_i * d1, m * MR)))
    Tec = Fraction(ceil_frac(Fraction(act_edges * d1 + n_act * d2, m * MR)))
    rtt_zc = gamma + (1 - gamma) * Fraction(act_edges, E_i)
    Tiz = ceil_frac(Fraction(lines, MR)) * rtt_zc
    return Tef, Tec, Tiz


def select_route(Tef: Fraction, Tec: Fraction, Tiz: Fraction,
                 alpha: Fraction = PAPER_ALPHA, beta: Fraction = PAPER_BETA) -> int:
    """Sec. V-A: C if Tec < alpha Tef and Tec < beta Tiz; else F if Tef < Tiz; else ZC."""
    if Tec < alpha * Tef and Tec < beta * Tiz:
        return ROUTE_C
    if Tef < Tiz:
        return ROUTE_F
    return ROUTE_Z


def plan(E_part: Sequence[int], n_act: Sequence[int], act_edges: Sequence[int],
         lines: Sequence[int], d1: int, resident: Optional[Iterable[int]] = None, **kw) -> List[int]:
    """Route of every partition for one iteration."""
    res = set(resident or ())
    alpha = kw.pop("alpha", PAPER_ALPHA)
    beta = kw.pop("beta", PAPER_BETA)
    out = []
    for i in range(len(E_part)):
        if int(act_edges[i]) == 0:
            out.append(ROUTE_NONE)
        elif i in res:
            out.append(ROUTE_CACHE)
        else:
            Tef, Tec, Tiz = costs(int(E_part[i]), int(act_edges[i]), int(n_act[i]), int(lines[i]),
                                  d1, **kw)
            out.append(select_route(Tef, Tec, Tiz, alpha, beta))
    return out


def combine_tasks(routes: Sequence[int], k: int = PAPER_K,
                  E_part: Optional[Sequence[int]] = None, cap_edges: Optional[int] = None
                  ) -> Tuple[List[List[int]], List[int], List[int], List[int]]:
    """Sec. V-B / Alg. 1 task combination.  Returns (F groups of consecutive
    partitions, C partitions, ZC partitions, cache partitions)."""
    groups: List[List[int]] = []
    cur: List[int] = []
    cur_edges = 0
    vc, vz, vcache = [], [], []
    for i, r in enumerate(routes):
        if r == ROUTE_F:
            e = int(E_part[i]) if E_part is not None else 0
            full = len(cur) >= k or (cap_edges is not None and cur and cur_edges + e > cap_edges)
            if full:
                groups.append(cur)
                cur, cur_edges = [], 0
            cur.append(i)
            cur_edges += e
        else:
            if cur:
                groups.append(cur)
                cur, cur_edges = [], 0
            if r == ROUTE_C:
                vc.append(i)
            elif r == ROUTE_Z:
                vz.append(i)
            elif r == ROUTE_CACHE:
                vcache.append(i)
    if cur:
        groups.append(cur)
    return groups, vc, vz, vcache


def hub_order(off: np.ndarray, dst: np.ndarray, frac: float = 0.08) -> List[int]:
    """Sec. VI-A hub sorting: the floor(frac * V) vertices with the largest
    H(v) = D_o(v) D_i(v) / (D_omax D_imax) first, in decreasing H (ties: smaller
    id first), then all other vertices in their natural order.  Returns perm
    with perm[new] = original id.  The normalising constant is positive and
    common to all vertices, so the order uses D_o(v) D_i(v) in exact integers."""
    V = len(off) - 1
    d_out = [int(off[v + 1]) - int(off[v]) for v in range(V)]
    d_in = [0] * V
    for x in dst.tolist():
        d_in[x] += 1
    k = int(frac * V)
    ranked = sorted(range(V), key=lambda v: (-(d_out[v] * d_in[v]), v))
    hubs = ranked[:k]
    chosen = set(hubs)
    return hubs + [v for v in range(V) if v not in chosen]


def relabel(off: np.ndarray, dst: np.ndarray, w, perm):
    """The CSR in the order perm (perm[new] = old): row new is old row perm[new]
    with every destination renamed to its new id."""
    V = len(off) - 1
    inv = np.empty(V, np.int64)
    inv[np.asarray(perm, np.int64)] = np.arange(V)
    deg = np.diff(off.astype(np.int64))[np.asarray(perm, np.int64)]
    off2 = np.concatenate([[0], np.cumsum(deg)]).astype(np.uint64)
    rows = [np.arange(int(off[o]), int(off[o + 1])) for o in perm]
    idx = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    dst2 = inv[dst.astype(np.int64)[idx]].astype(np.uint32)
    w2 = None if w is None else w[idx]
    return off2, dst2, w2
