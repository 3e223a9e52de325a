"""Continuous-batching query server over the hytg serving ABI.

One engine (hytg context with its own copy of the graph) per algorithm;
each engine runs one batched run whose slots hold queries.  The loop admits
arrived queries at iteration boundaries, steps every engine that has busy
slots (one iteration each, interleaved, so the engines' device work
overlaps), and retires converged queries.  Admission is by device memory:
each engine's budget holds its edge-side data and its queries' state in
frames of 8 queries, so a query is admitted only into a free slot whose
group already has a frame, or whose group can take a free frame; otherwise
it waits until a finished query gives memory back, even when slots are free.

`python -m paper_2208_14935_gb300.serve` runs the serving benchmark on a
synthetic graph and prints one JSON line.
"""
from __future__ import annotations

import argparse
import collections
import json
import os
import sys
import threading
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import hytg


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    algo: str               # "bfs", "sssp" or "ppr"
    source: int
    admitted: float = -1.0
    done: float = -1.0
    result: Optional[np.ndarray] = None


@dataclass
class _Lane:
    eng: "hytg.Engine"
    algo: str
    slots: int
    occupant: List[Optional[Request]] = field(default_factory=list)
    waiting: collections.deque = field(default_factory=collections.deque)
    steps: int = 0
    memory_waits: int = 0          # admissions refused for lack of a free frame
    max_busy: int = 0              # most queries on the device at once


class Server:
    """Serve BFS/SSSP/PPR queries with continuous batching.

    threads=False: one host thread steps the engines in turn.  threads=True:
    one host thread per engine (the ctypes calls release the interpreter
    lock), so one engine's host-side waits do not hold back the others."""

    def __init__(self, engines: Dict[str, "hytg.Engine"], slots: Optional[Dict[str, int]] = None,
                 keep_results: bool = True, threads: bool = False):
        self.lanes: Dict[str, _Lane] = {}
        self.keep_results = keep_results
        self.threads = threads
        for algo, eng in engines.items():
            n = (slots or {}).get(algo, 32 if algo == "ppr" else 64)
            lane = _Lane(eng, algo, n, [None] * n)
            self.lanes[algo] = lane

    FRAME = 8                      # slots [8 g, 8 g + 8) share one frame of device memory

    def _admit(self, lane: _Lane, t0: float, clock) -> None:
        """Free slots of groups that already hold a frame first (no new
        memory), then slots of empty groups while the engine has a free frame."""
        if not lane.waiting:
            return
        F = self.FRAME
        groups = range((lane.slots + F - 1) // F)
        framed = [any(lane.occupant[g * F:(g + 1) * F]) for g in groups]
        order = ([s for g in groups if framed[g] for s in range(g * F, min((g + 1) * F, lane.slots))] +
                 [s for g in groups if not framed[g] for s in range(g * F, min((g + 1) * F, lane.slots))])
        memory_full = False
        for s in order:
            if not lane.waiting:
                break
            g = s // F
            if lane.occupant[s] is not None or (memory_full and not framed[g]):
                continue
            r = lane.waiting[0]
            try:
                hytg.hytg_serve_admit(lane.eng.ctx, s, r.source)
            except hytg.HytgError as ex:
                if ex.status != hytg.HYTG_ERR_BUDGET:
                    raise
                memory_full = True          # no free frame: the query waits for memory
                lane.memory_waits += 1
                continue
            lane.waiting.popleft()
            framed[g] = True
            r.admitted = clock() - t0
            lane.occupant[s] = r
        lane.max_busy = max(lane.max_busy, sum(o is not None for o in lane.occupant))

    def _step(self, lane: _Lane, t0: float, clock) -> List[Request]:
        """One iteration of the lane's engine; returns the queries it finished."""
        fin, _ = hytg.hytg_serve_step(lane.eng.ctx)
        lane.steps += 1
        out = []
        s = 0
        while fin:
            if fin & 1:
                r = lane.occupant[s]
                res = hytg.hytg_serve_fetch(lane.eng.ctx, s, lane.eng.V, hytg.ALGOS[lane.algo])
                r.done = clock() - t0
                if self.keep_results:
                    r.result = res
                lane.occupant[s] = None
                out.append(r)
            fin >>= 1
            s += 1
        return out

    def run(self, requests: List[Request], clock=time.perf_counter) -> List[Request]:
        for lane in self.lanes.values():
            hytg.hytg_serve_begin(lane.eng.ctx, hytg.ALGOS[lane.algo], lane.slots)
        todo = collections.deque(sorted(requests, key=lambda r: r.arrival))
        t0 = clock()
        try:
            if self.threads:
                return self._run_threaded(todo, t0, clock)
            done: List[Request] = []
            while todo or any(l.waiting or any(l.occupant) for l in self.lanes.values()):
                now = clock() - t0
                while todo and todo[0].arrival <= now:
                    r = todo.popleft()
                    self.lanes[r.algo].waiting.append(r)
                busy = False
                for lane in self.lanes.values():
                    self._admit(lane, t0, clock)
                    if any(lane.occupant):
                        busy = True
                        done.extend(self._step(lane, t0, clock))
                if not busy and todo:
                    wait = todo[0].arrival - (clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
            return done
        finally:
            for lane in self.lanes.values():
                hytg.hytg_serve_end(lane.eng.ctx)

    def _run_threaded(self, todo: collections.deque, t0: float, clock) -> List[Request]:
        lock = threading.Lock()
        done: List[Request] = []
        left = collections.Counter(r.algo for r in todo)     # not yet admitted, per engine
        errors: List[BaseException] = []

        def lane_loop(lane: _Lane) -> None:
            try:
                while True:
                    with lock:
                        now = clock() - t0
                        while todo and todo[0].arrival <= now:
                            r = todo.popleft()
                            self.lanes[r.algo].waiting.append(r)
                        before = len(lane.waiting)
                        self._admit(lane, t0, clock)
                        left[lane.algo] -= before - len(lane.waiting)
                        busy = any(lane.occupant)
                        finished = not busy and left[lane.algo] == 0
                        nxt = todo[0].arrival if todo else None
                    if finished:
                        return
                    if busy:
                        out = self._step(lane, t0, clock)
                        if out:
                            with lock:
                                done.extend(out)
                    elif nxt is not None:
                        wait = nxt - (clock() - t0)
                        time.sleep(min(max(wait, 0.0), 0.01) if wait > 0 else 0.0005)
                    else:
                        time.sleep(0.0005)
            except BaseException as ex:             # surfaced after the join
                errors.append(ex)

        workers = [threading.Thread(target=lane_loop, args=(lane,)) for lane in self.lanes.values()]
        for w in workers:
            w.start()
        for w in workers:
            w.join()
        if errors:
            raise errors[0]
        return done


def latency_stats(done: List[Request]) -> Dict[str, float]:
    lat = np.array([r.done - r.arrival for r in done])
    span = max(r.done for r in done) - min(r.arrival for r in done)
    return {"n": len(done), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "qps": len(done) / span if span > 0 else float("nan")}


def poisson_requests(n: int, rate: float, sources: Dict[str, np.ndarray], mix=(("bfs", 2), ("sssp", 2), ("ppr", 1)),
                     seed: int = 1) -> List[Request]:
    """n requests with exponential inter-arrival times (Poisson process of the
    given rate, queries/s), algorithms drawn in the ratio `mix`, sources drawn
    from `sources[algo]`; rate = inf gives a burst at t = 0."""
    rng = np.random.default_rng(seed)
    algos = [a for a, w in mix for _ in range(w)]
    t = 0.0
    out = []
    for i in range(n):
        if np.isfinite(rate):
            t += rng.exponential(1.0 / rate)
        a = algos[rng.integers(len(algos))]
        out.append(Request(i, t, a, int(rng.choice(sources[a]))))
    return out


def _main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--graph", default="chunglu", choices=["chunglu", "rmat"])
    ap.add_argument("--log2v", type=int, default=26)
    ap.add_argument("--log2e", type=int, default=31)
    ap.add_argument("--budget-gb", type=float, default=16.0,
                    help="device budget of the whole server (10^9 bytes), split among the engines")
    ap.add_argument("--shares", default="0.265,0.265,0.47",
                    help="fractions of the budget for the BFS, SSSP and PPR engines")
    ap.add_argument("--n", type=int, default=200, help="requests per rate")
    ap.add_argument("--rates", default="0.25,0.5,0.9", help="fractions of the saturation rate")
    ap.add_argument("--threads", action="store_true", help="one host thread per engine")
    ap.add_argument("--both", action="store_true",
                    help="run the rated sequence with one host thread and then with one per engine")
    ap.add_argument("--max-seconds", type=float, default=60.0,
                    help="cap on the arrival span of each rated run (fewer requests at low rates)")
    args = ap.parse_args()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from gen import graphgen as gg
    from . import build as bld
    bld.build()
    t = time.perf_counter()
    if args.graph == "chunglu":
        g = gg.chung_lu(1 << args.log2v, 1 << args.log2e, beta=2.1, wmax=255, seed=1)
    else:
        g = gg.rmat(args.log2v, edge_factor=1 << (args.log2e - args.log2v), seed=1)
    gen_s = time.perf_counter() - t
    budget = int(args.budget_gb * 1e9)
    # the total budget is split among the three engines: each holds its own
    # edge-side data and its queries' frames (8 queries each: BFS/SSSP V * 32
    # bytes, PPR V * 96 bytes).  The edge side needs at least one staging slot
    # of the largest partition; on the power-law graphs the first partition
    # (32 hub vertices, one bitmap word) holds about 9 % of the edges.  The
    # default split gives 2^26 vertices and 2^31 edges in 16e9 bytes one
    # frame per engine (8 queries each) beside that slot.
    shares = {a: float(x) for a, x in zip(("bfs", "sssp", "ppr"), args.shares.split(","))}
    tot = sum(shares.values())
    engines = {}
    unweighted = gg.CSR(g.V, g.E, g.off, g.dst, None, g.name)
    for algo in ("bfs", "sssp", "ppr"):
        e = hytg.Engine(params={"part_bytes": 4 * 1024 * 1024})
        e.load(g if algo == "sssp" else unweighted)
        e.set_budget(int(budget * shares[algo] / tot))
        engines[algo] = e
    cand = np.flatnonzero(np.diff(g.off.astype(np.int64)) > 0)
    rng = np.random.default_rng(3)
    pools = {a: rng.choice(cand, 4096, replace=True) for a in ("bfs", "sssp", "ppr")}
    out = {"metric": "served queries: p50/p99 latency and queries/s (continuous batching)",
           "graph": {"family": args.graph, "V": g.V, "E": g.E, "gen_s": round(gen_s, 1)},
           "budget_bytes": budget, "mix": "BFS:SSSP:PPR = 2:2:1", "slots": {"bfs": 64, "sssp": 64, "ppr": 32},
           "engine_budget_bytes": {a: int(budget * shares[a] / tot) for a in shares}, "runs": []}
    for threads in ([False, True] if args.both else [args.threads]):
        srv = Server(engines, keep_results=False, threads=threads)
        # saturation: every request present at t = 0 (closed burst)
        warm = poisson_requests(min(64, args.n), float("inf"), pools, seed=9)
        srv.run(warm)
        sat_reqs = poisson_requests(args.n, float("inf"), pools, seed=10)
        sat = latency_stats(srv.run(sat_reqs))
        if "frames" not in out:
            mem = {}
            for lane in srv.lanes.values():
                hytg.hytg_serve_begin(lane.eng.ctx, hytg.ALGOS[lane.algo], lane.slots)
                mem[lane.algo] = hytg.hytg_serve_get_info(lane.eng.ctx)
                hytg.hytg_serve_end(lane.eng.ctx)
            out["frames"] = {a: {"frames": m["frames"], "frame_bytes": m["frame_bytes"],
                                 "queries_at_once": m["frames"] * m["slots_per_frame"],
                                 "edge_budget_bytes": m["edge_budget_bytes"]} for a, m in mem.items()}
        run = {"host_threads": 3 if threads else 1, "saturation": sat, "rates": {}}
        for frac in [float(x) for x in args.rates.split(",")]:
            rate = frac * sat["qps"]
            n = max(8, min(args.n, int(rate * args.max_seconds)))
            reqs = poisson_requests(n, rate, pools, seed=int(frac * 1000))
            run["rates"][f"{frac:g}x"] = {"offered_qps": rate, **latency_stats(srv.run(reqs))}
        run["memory_waits"] = {a: l.memory_waits for a, l in srv.lanes.items()}
        run["max_busy"] = {a: l.max_busy for a, l in srv.lanes.items()}
        out["runs"].append(run)
    print(json.dumps(out), flush=True)
    for e in engines.values():
        e.close()


if __name__ == "__main__":
    _main()
