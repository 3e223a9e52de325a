"""Benchmark: GTEPS of the hybrid-transfer engine at a capped device budget.

Workload (one "step"): on an R-MAT scale-24 graph (16,777,216 vertices,
268,435,456 directed edges, a=0.57 b=0.19 c=0.19 d=0.05, seed 1, uint32
weights uniform in [1, 64]) whose edge arrays live in pinned host memory,
with a device budget of 25 % of the graph bytes: BFS and SSSP from vertex 0,
connected components on the symmetrised graph (536,870,912 edges) and
delta-PageRank (damping 0.85, FP32 residual threshold 1e-9), each to
convergence through the C ABI.

value  = edges relaxed (sum over iterations of the active out-edges, the
         algorithmic count, identical for every route) / device time of the
         runs (CUDA events on the library's main stream, which joins all of
         its streams), summed over the K timed steps, over all ranks, divided
         by the slowest rank's time.  Second-pass re-relaxations over resident
         partitions (Sec. VI-A) depend on the schedule and are reported beside
         it (config.gteps_with_second_pass), not in it;
e2e    = the same edges over host wall time of hytg_run + hytg_fetch_result
         (the public calls), including the result copies to host memory.
The host-link denominator is the pinned-memcpy probe measured in the same
process before and after the timed steps (their mean).

Multi-GPU: replicas only (each rank runs the whole workload on its own GPU;
no data-path collective); the barrier and max-over-ranks timing use
torch.distributed.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GTEPS at capped device budget; host-link GB/s % of measured; batched vs plain"
ALGOS = ["bfs", "sssp", "cc", "pagerank"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=24)
    ap.add_argument("--budget-frac", type=float, default=0.25)
    ap.add_argument("--part-bytes", type=float, default=4 * 1024 * 1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-timing", action="store_true", help="skip per-kernel CUDA events")
    ap.add_argument("--param", action="append", default=[], help="key=value engine parameter")
    ap.add_argument("--algos", default=",".join(ALGOS),
                    help="comma-separated subset of bfs,sssp,cc,pagerank (profiling runs)")
    ap.add_argument("--no-probe", action="store_true", help="skip the host-link probe")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain runs")
    ap.add_argument("--timeline-out", default="", metavar="PATH",
                    help="save each algorithm's launch timeline of the last timed step (numpy .npz); "
                         "with --param device_loop=0 its k_second_pass/k_relax entries follow the "
                         "process's launch order, so a profiler's launch index maps to an edge count")
    ap.add_argument("--mesh-only", type=int, default=0, metavar="SIDE",
                    help="only the high-diameter workload: SIDE x SIDE 4-neighbour mesh with 0.1 %% "
                         "local shortcuts, weights in [1, 1000], 20 %% budget; BFS, SSSP, CC from "
                         "vertex 0 (with and without the device loop); prints its own line")
    ap.add_argument("--autotune", action="store_true",
                    help="with --batched-only: tune partition size, F-task width and MR on the "
                         "batched BFS/SSSP runs first (paper_2208_14935_gb300.autotune)")
    ap.add_argument("--batched-only", type=int, default=0, metavar="SCALE",
                    help="only the batched workload (64 BFS/SSSP sources, 32 PPR seeds) on R-MAT "
                         "SCALE against the same sources run one at a time; prints its own line")
    return ap.parse_args()


# --------------------------------------------------------------- helpers --
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(local_units: float, local_ms: float, world: int, group=None):
    """Whole-job throughput over ranks: sum of units / max of times."""
    if world == 1:
        return local_units, local_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_units], dtype=torch.float64)
    m = torch.tensor([local_ms], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t, m = t.cuda(), m.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(m, op=dist.ReduceOp.MAX, group=group)
    return float(t.item()), float(m.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def make_graphs(scale):
    from gen import graphgen as gg
    g = gg.rmat(scale, seed=1, wmax=64)
    s = gg.symmetrize(g)
    return g, s


def batched_vs_plain(hytg, eng, g, n_plain_sssp=16, n_plain_ppr=4):
    """Batched runs (64 BFS sources, 64 SSSP sources, 32 PPR seeds, seeded
    draws among vertices with out-edges) against the same sources run one at a
    time, on the same engine, graph and budget.  `speedup` is the time to
    solution per source, plain over batched (device time, CUDA events).  The
    rate is per-source edges relaxed / device time; for BFS and SSSP the edge
    counts are fixed by the graph, so the two ratios agree, while PPR's count
    depends on the schedule (an iteration pushes whatever residual each seed
    holds) and only the time ratio compares like with like.  For PPR the line
    also gives the seed updates per second, second pass included, against the
    frame-push probe (8 seeds per vertex and edge, with vector reductions)."""
    rng = np.random.default_rng(7)
    cand = np.flatnonzero(np.diff(g.off.astype(np.int64)) > 0)
    out = {}
    for algo, k, n_plain in (("bfs", 64, 64), ("sssp", 64, n_plain_sssp), ("ppr", 32, n_plain_ppr)):
        src = rng.choice(cand, k, replace=False).tolist()
        a = hytg.ALGOS[algo]
        hytg.hytg_run(eng.ctx, a, src)                       # warm-up
        b_ms, b_edges, b_extra = 0.0, 0, 0
        for _ in range(2):
            hytg.hytg_run(eng.ctx, a, src)
            st = eng.stats()
            b_ms += st["device_ms"]
            b_edges += st["source_edges"]
            b_extra += st["extra_edges"]
        p_ms, p_edges = 0.0, 0
        for v in src[:n_plain]:
            hytg.hytg_run(eng.ctx, a, [v])
            st = eng.stats()
            p_ms += st["device_ms"]
            p_edges += st["edges_relaxed"]
        bg = b_edges / (b_ms * 1e-3) / 1e9
        pg = p_edges / (p_ms * 1e-3) / 1e9
        per_src_b = b_ms / 2 / k
        per_src_p = p_ms / n_plain
        out[algo] = {"sources": k, "batched_gteps": bg, "batched_ms": b_ms / 2,
                     "batched_ms_per_source": per_src_b,
                     "plain_gteps": pg, "plain_ms_per_source": per_src_p,
                     "plain_sources_timed": n_plain,
                     "speedup": per_src_p / per_src_b if per_src_b else None,
                     "gteps_ratio": bg / pg if pg else None}
        if algo == "ppr":
            upd = (b_edges + b_extra) / (b_ms * 1e-3) / 1e9
            roof = {w: hytg.hytg_probe_frame_push(eng.ctx, 1 << 26, 3, w) for w in (1, 4)}
            out[algo]["seed_updates_g_per_s"] = upd
            out[algo]["frame_push_probe_g_per_s"] = {"scalar": roof[1], "v4": roof[4]}
            out[algo]["frac_of_v4_probe_dense"] = upd / (8 * roof[4]) if roof[4] else None
    return out


# ------------------------------------------------------- reference arm ----
def oracle_sample(name, g, s):
    """One oracle run on the host cores (plain single-threaded C) on the full
    graph: FIFO BFS or Dijkstra from vertex 0, union-find CC on the
    symmetrised graph, or one FP64 power-iteration sweep of PageRank (the full
    solve takes over a hundred sweeps).  Returns (edges processed, seconds)."""
    from oracle import oracle as orc
    t0 = time.perf_counter()
    if name == "bfs":
        _, e = orc.bfs(g, 0)
    elif name == "sssp":
        _, e, _ = orc.sssp(g, 0)
    elif name == "cc":
        orc.cc(s)
        e = s.E
    else:
        orc.pagerank(g, maxit=1)
        e = g.E
    return int(e), time.perf_counter() - t0


ORACLE_WHAT = {"bfs": "FIFO BFS from vertex 0", "sssp": "Dijkstra from vertex 0",
               "cc": "union-find CC on the symmetrised graph",
               "pagerank": "one FP64 PageRank power-iteration sweep"}


def cpu_oracle_samples(g, s, algos, budget_s: float = 25.0):
    """Each algorithm of the step once through the oracle, while the budget lasts."""
    out, used = {}, 0.0
    for a in algos:
        if used > budget_s:
            break
        e, dt = oracle_sample(a, g, s)
        used += dt
        out[a] = {"edges": e, "s": round(dt, 3), "gteps": e / dt / 1e9, "what": ORACLE_WHAT[a]}
    return out


def step_config(args, g, s, algos, world):
    """The bench step's `config`, shared by both arms."""
    graph_bytes = g.E * 8 + (g.V + 1) * 8
    sym_bytes = s.E * 4 + (s.V + 1) * 8
    return {"workload": f"rmat{args.scale} {'+'.join(algos)}, edges in pinned host memory, "
                        f"budget {args.budget_frac:.0%} of graph bytes",
            "V": g.V, "E": g.E, "E_sym": s.E, "budget_bytes": int(args.budget_frac * graph_bytes),
            "budget_bytes_cc": int(args.budget_frac * sym_bytes),
            "part_bytes": args.part_bytes, "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (edge arrays in host memory)"}


def run_reference(args):
    """The oracle as the CPU reference: every step runs one algorithm of the
    GPU step on the full graph, in turn (BFS, Dijkstra, union-find CC, one
    PageRank sweep), so the timed steps sample all four; value = edges
    processed / seconds over the timed steps."""
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    g, s = make_graphs(args.scale)
    from oracle import oracle as orc
    orc.build()
    algos = [a for a in args.algos.split(",") if a]
    total_e, total_s = 0, 0.0
    per = {}
    for i in range(args.warmup + args.steps):
        a = algos[(i - args.warmup) % len(algos)]
        e, dt = oracle_sample(a, g, s)
        if i >= args.warmup:
            total_e += e
            total_s += dt
            p = per.setdefault(a, {"edges": 0, "s": 0.0, "steps": 0})
            p["edges"] += e
            p["s"] += dt
            p["steps"] += 1
    v = total_e / total_s / 1e9
    for p in per.values():
        p["gteps"] = p["edges"] / p["s"] / 1e9
    sample = ("oracle (single-threaded C) on the full graph, one algorithm per step in turn: " +
              ", ".join(ORACLE_WHAT[a] for a in algos))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32 (PageRank f64)",
            "data": "synthetic",
            "config": step_config(args, g, s, algos, 1),
            "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": sample, "per_algo": per, "host_cores": os.cpu_count()},
            "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- ours ----
def run_batched_only(args):
    """Batched workload at its own size (R-MAT 25: 33,554,432 vertices,
    536,870,912 edges, 25 % budget): 64 BFS and SSSP sources and 32 PPR
    seeds per run, against the same sources one at a time."""
    from paper_2208_14935_gb300 import build as bld
    bld.build()
    from paper_2208_14935_gb300 import hytg
    from gen import graphgen as gg
    t0 = time.perf_counter()
    g = gg.rmat(args.batched_only, seed=1, wmax=64)
    t_gen = time.perf_counter() - t0
    graph_bytes = g.E * 8 + (g.V + 1) * 8
    eng = hytg.Engine(g, budget=int(args.budget_frac * graph_bytes),
                      params={"part_bytes": args.part_bytes})
    tuned = None
    if args.autotune:
        from paper_2208_14935_gb300.autotune import autotune
        rng = np.random.default_rng(5)
        cand = np.flatnonzero(np.diff(g.off.astype(np.int64)) > 0)
        src = rng.choice(cand, 64, replace=False).tolist()
        space = {"part_bytes": [2 << 20, 4 << 20, 8 << 20], "k": [2, 4, 8], "MR": [64, 256, 1024]}
        t0 = time.perf_counter()
        tuned = autotune(eng, [("bfs", src), ("sssp", src)], space=space, reps=1)
        tuned = {"params": tuned, "seconds": round(time.perf_counter() - t0, 1),
                 "workload": "64-source batched BFS + SSSP (other sources than the measured ones)"}
    res = batched_vs_plain(hytg, eng, g)
    eng.close()
    line = {"metric": "batched vs plain GTEPS (per-source edges relaxed / device time)",
            "unit": "GTEPS", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"rmat{args.batched_only} batched BFS/SSSP x64, PPR x32, budget "
                                   f"{args.budget_frac:.0%} of graph bytes",
                       "V": g.V, "E": g.E, "budget_bytes": int(args.budget_frac * graph_bytes),
                       "graph_gen_s": round(t_gen, 1)},
            "autotuned": tuned, "batched_vs_plain": res}
    print(json.dumps(line), flush=True)


def run_mesh_only(args):
    """The road-like workload: long tails of tiny frontiers, where the
    per-iteration cost (planning + launches) rather than the link decides."""
    from paper_2208_14935_gb300 import build as bld
    bld.build()
    from paper_2208_14935_gb300 import hytg
    from gen import graphgen as gg
    t0 = time.perf_counter()
    g = gg.mesh(args.mesh_only, args.mesh_only, shortcut_frac=0.001, radius=16, seed=1, wmax=1000)
    t_gen = time.perf_counter() - t0
    graph_bytes = g.E * 8 + (g.V + 1) * 8
    eng = hytg.Engine(g, budget=int(0.2 * graph_bytes), params={"part_bytes": args.part_bytes})
    res = {}
    for loop in (1, 0):
        eng.set_param("device_loop", loop)
        for algo in ("bfs", "sssp", "cc"):
            hytg.hytg_run(eng.ctx, hytg.ALGOS[algo], None if algo == "cc" else [0])
            st = eng.stats()
            res[f"{algo}{'' if loop else '_host_loop'}"] = {
                "ms": round(st["device_ms"], 1), "iterations": st["iterations"],
                "graph_iterations": st["graph_iterations"], "edges_relaxed": st["edges_relaxed"],
                "gteps": st["edges_relaxed"] / (st["device_ms"] * 1e-3) / 1e9,
                "us_per_iteration": round(st["device_ms"] * 1e3 / max(1, st["iterations"]), 1)}
    eng.close()
    line = {"metric": "mesh BFS/SSSP/CC device time (long tails of tiny frontiers)", "unit": "ms",
            "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"mesh {args.mesh_only}x{args.mesh_only}, 0.1% shortcuts, budget 20% "
                                   "of graph bytes", "V": g.V, "E": g.E,
                       "budget_bytes": int(0.2 * graph_bytes), "graph_gen_s": round(t_gen, 1)},
            "runs": res}
    print(json.dumps(line), flush=True)


U64_MAX = (1 << 64) - 1
LINK_KINDS = (5, 7, 8)          # C gathers, Z relaxes, F copies: the launches that move host-link bytes


def union_ms(iv):
    """Total length of the union of intervals [(start, end), ...]."""
    busy, lo, hi = 0.0, 0.0, -1.0
    for a, b in sorted(iv):
        if a > hi:
            if hi > lo:
                busy += hi - lo
            lo, hi = a, b
        elif b > hi:
            hi = b
    if hi > lo:
        busy += hi - lo
    return busy


def copy_boundaries(tl, min_gap_ms=0.1):
    """The F copies' share of a run: the time the copy engine was busy (union
    of the copy intervals) and the idle stretches between copies.  Copies
    of one iteration run back to back, a few microseconds apart; a stretch
    longer than min_gap_ms is mostly the boundary between two iterations
    that copy (the last tasks' relaxes, then the next planning), sometimes a
    copy waiting for its staging slot.  Returns the busy time, the number of
    such stretches and their mean length."""
    cp = tl["kind"] == 8
    order = np.argsort(tl["start_ms"][cp], kind="stable")
    cs, ce = tl["start_ms"][cp][order], tl["end_ms"][cp][order]
    gaps, end = [], None
    for a, b in zip(cs, ce):
        if end is not None and a - end > min_gap_ms:
            gaps.append(float(a - end))
        end = b if end is None else max(end, b)
    return {"copy_busy_ms": union_ms(list(zip(cs, ce))), "idle_stretches": len(gaps),
            "idle_stretch_ms": float(np.mean(gaps)) if gaps else None}


def timeline_summary(tl, hytg):
    """Per-run figures from the launch timeline: every F copy's rate, the wall
    time during which any route moved host-link bytes, per-launch edge
    counts and durations of the two PageRank kernels, and the copies' share
    of each iteration (copy_boundaries)."""
    dur = tl["end_ms"] - tl["start_ms"]
    cp = tl["kind"] == 8
    link = np.isin(tl["kind"], LINK_KINDS)
    sp = (tl["kind"] == hytg.K_SECOND_PASS) & (tl["edges"] != U64_MAX)
    rf = tl["kind"] == 4
    return {"copy_gbs": (tl["bytes"][cp] / np.maximum(dur[cp], 1e-6) / 1e6).tolist(),
            "copy_stream": tl["stream"][cp].tolist(),
            "link_busy_ms": union_ms(list(zip(tl["start_ms"][link], tl["end_ms"][link]))),
            "sp_n": int(sp.sum()), "sp_ms": float(dur[sp].sum()), "sp_edges": int(tl["edges"][sp].sum()),
            "sp_vertices": int(tl["vertices"][sp].sum()),
            "rf_n": int(rf.sum()), "rf_ms": float(dur[rf].sum()), "rf_edges": int(tl["edges"][rf].sum()),
            **copy_boundaries(tl)}


def pct(xs, q):
    return float(np.percentile(xs, q)) if len(xs) else None


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.batched_only:
        return run_batched_only(args)
    if args.mesh_only:
        return run_mesh_only(args)
    rank, world, local = dist_env()
    algos = [a for a in args.algos.split(",") if a]
    assert all(a in ALGOS for a in algos), args.algos
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_2208_14935_gb300 import build as bld
    bld.build()
    from paper_2208_14935_gb300 import hytg
    t_gen = time.perf_counter()
    g, s = make_graphs(args.scale)
    t_gen = time.perf_counter() - t_gen
    graph_bytes = g.E * 8 + (g.V + 1) * 8
    sym_bytes = s.E * 4 + (s.V + 1) * 8
    params = {"part_bytes": args.part_bytes, "timing": 0 if args.no_timing else 1}
    for kv in args.param:
        k, v = kv.split("=")
        params[k] = float(v)
    eng = hytg.Engine(g, budget=int(args.budget_frac * graph_bytes), device=local, params=params)
    eng_s = hytg.Engine(s, budget=int(args.budget_frac * sym_bytes), device=local, params=params)
    damping = eng.get_param("pr_damping")

    def one_step():
        per = {}
        for algo in algos:
            e = eng_s if algo == "cc" else eng
            src = 0 if algo in ("bfs", "sssp") else None
            t0 = time.perf_counter()
            hytg.hytg_run(e.ctx, hytg.ALGOS[algo], None if src is None else [src])
            out = hytg.hytg_fetch_result(e.ctx, e.V, hytg.ALGOS[algo])
            wall = (time.perf_counter() - t0) * 1e3
            st = e.stats()
            raw = e.timeline() if not args.no_timing else None
            tl = timeline_summary(raw, hytg) if raw is not None else None
            per[algo] = {"stats": st, "wall_ms": wall, "d2h": out.nbytes,
                         "h2d": 0 if src is None else 4, "tl": tl}
            if args.timeline_out:
                per[algo]["tl_raw"] = raw
        return per

    # the link denominator, measured in this process before and after the timed steps
    probe_before = None if args.no_probe else eng.probe_link(1 << 30, 10)
    for _ in range(args.warmup):
        one_step()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    steps = [one_step() for _ in range(args.steps)]
    barrier(world)
    clk = clocks.stop()
    probe_after = None if args.no_probe else eng.probe_link(1 << 30, 10)
    batched = None if args.no_batched else batched_vs_plain(hytg, eng, g)
    red_probe = None if args.no_probe else eng.probe_atomics(1 << 28, 5)
    # the PageRank kernels' own target pattern: R-MAT in-degree skew after hub
    # sorting, pushes to the first hub_replicas ids into per-SM replicas
    hub_probe = None if args.no_probe else hytg.hytg_probe_atomics_hub(
        eng.ctx, 1 << 28, 5, int(eng.get_param("hub_replicas")))
    probe = float("nan") if args.no_probe else (probe_before[0] + probe_after[0]) / 2
    if args.timeline_out and rank == 0:
        np.savez(args.timeline_out, **{a: steps[-1][a]["tl_raw"] for a in algos if "tl_raw" in steps[-1][a]})

    def tot(a, key, i=None):
        return sum((p[a]["stats"][key] if i is None else p[a]["stats"][key][i]) for p in steps)

    # TEPS numerator: active out-edges relaxed over the iterations (the
    # algorithmic count, the same for every route); second-pass re-relaxations
    # over resident partitions are reported beside it, not in it
    edges = sum(tot(a, "edges_relaxed") for a in algos)
    extra = sum(tot(a, "extra_edges") for a in algos)
    dev_ms = sum(tot(a, "device_ms") for a in algos)
    wall_ms = sum(p[a]["wall_ms"] for p in steps for a in algos)
    launches = sum(tot(a, "kernel_launches") for a in algos)
    tot_edges, max_ms = aggregate(float(edges), dev_ms, world)
    tot_edges_w, max_wall = aggregate(float(edges), wall_ms, world)
    value = tot_edges / (max_ms * 1e-3) / 1e9
    e2e = tot_edges_w / (max_wall * 1e-3) / 1e9

    # host link: F bytes copied, C/Z sectors the kernels read from host memory
    link_bytes = sum(tot(a, "link_sector_bytes", r) for a in algos for r in range(5))
    model_bytes = sum(tot(a, "link_bytes", r) for a in algos for r in range(5))
    per_route = {}
    for r, name in ((2, "F"), (3, "C"), (4, "Z")):
        b = sum(tot(a, "link_sector_bytes", r) for a in algos)
        busy = sum(tot(a, "route_busy_ms", r) for a in algos)
        per_route[name] = {"bytes": b, "model_line_bytes": sum(tot(a, "link_bytes", r) for a in algos),
                           "busy_ms": round(busy, 2),
                           "frac_of_probe": (b / (busy * 1e-3) / 1e9 / probe) if busy > 0 else None}
    per_algo = {}
    for a in algos:
        ed, ms = tot(a, "edges_relaxed"), tot(a, "device_ms")
        ex = tot(a, "extra_edges")
        lb = sum(tot(a, "link_sector_bytes", r) for r in range(5))
        st = steps[-1][a]["stats"]
        d = {"gteps": ed / (ms * 1e-3) / 1e9, "ms": round(ms / len(steps), 2),
             "link_gbs": lb / (ms * 1e-3) / 1e9, "link_frac": lb / (ms * 1e-3) / 1e9 / probe,
             "iterations": st["iterations"], "graph_iterations": st["graph_iterations"],
             "edges_relaxed": st["edges_relaxed"]}
        if ex:
            d["second_pass_edges"] = st["extra_edges"]
            d["gteps_with_second_pass"] = (ed + ex) / (ms * 1e-3) / 1e9
        if not args.no_timing:
            busy = sum(p[a]["tl"]["link_busy_ms"] for p in steps)
            d["link_busy_frac"] = busy / ms
            d["link_frac_while_busy"] = lb / (busy * 1e-3) / 1e9 / probe if busy > 0 else None
            # the copy engine's share of the run and its idle stretches
            # (mostly the boundaries of the iterations that copy)
            d["copy_busy_frac"] = sum(p[a]["tl"]["copy_busy_ms"] for p in steps) / ms
            d["copy_idle_stretches"] = steps[-1][a]["tl"]["idle_stretches"]
            gaps = [p[a]["tl"]["idle_stretch_ms"] for p in steps if p[a]["tl"]["idle_stretch_ms"] is not None]
            d["copy_idle_stretch_ms"] = float(np.mean(gaps)) if gaps else None
        if a == "pagerank":
            # a-posteriori bound on the L1 error of the normalised ranks:
            # sum |delta| left / ((1 - d) * sum rank)
            d["l1_bound"] = st["pr_residual_sum"] / ((1 - damping) * st["pr_rank_sum"])
        per_algo[a] = d

    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    roofline, roofline_l2 = None, None
    if not args.no_timing and "pagerank" in algos:
        # PageRank is most of the step; its two heaviest kernels are the second
        # pass over resident partitions and the F-route relax.  Per launch from
        # the timeline (CUDA events on the launching stream, timed region only).
        tls = [p["pagerank"]["tl"] for p in steps]
        prs = [p["pagerank"]["stats"] for p in steps]
        sp_n, sp_ms = sum(t["sp_n"] for t in tls), sum(t["sp_ms"] for t in tls)
        sp_e, sp_v = sum(t["sp_edges"] for t in tls), sum(t["sp_vertices"] for t in tls)
        rf_n, rf_ms = sum(t["rf_n"] for t in tls), sum(t["rf_ms"] for t in tls)
        rf_e = sum(t["rf_edges"] for t in tls)
        rf_v = sum(st["route_vertices"][2] for st in prs)
        kern = {}
        if sp_n:
            # per relaxed edge 4 B edge + 8 B value read-modify-write; per
            # scanned vertex 16 B offsets, 4 B delta read, 8 B delta and rank updates
            kern["k_second_pass<PageRank>"] = (sp_n, sp_ms, sp_e, sp_e * 12 + sp_v * 28,
                                               "per edge 4 + 8 (value RMW), per scanned vertex 28",
                                               sp_v)
        if rf_n:
            # per edge 4 B edge + 8 B RMW, per list entry 20 B
            kern["k_relax<PageRank> F route"] = (rf_n, rf_ms, rf_e, rf_e * 12 + rf_v * 20,
                                                 "per edge 4 + 8 (value RMW), per active vertex 20",
                                                 rf_v)
        if kern:
            dom = max(kern, key=lambda k: kern[k][1])
            n, ms, e_, alg, model, vv = kern[dom]
            achieved = alg / (ms * 1e-3) / 1e9
            traffic, note = None, "no ncu DRAM capture of the current kernel"
            if dom.startswith("k_second_pass"):
                # DRAM bytes from one cold-cache ncu capture of each of its two
                # launches on R-MAT 22: the push read 29.8 MB for 4,183,639
                # edges, the take 0.43 MB for 22,240 vertices; scaled to this
                # run's mean launch by its edges and vertices
                traffic = (29.778176e6 / 4183639) * (e_ / n) + (430592.0 / 22240) * (vv / n)
                note = ("scaled from ncu captures on R-MAT 22 (push 7.12 B/edge, take 19.4 B/vertex, "
                        "cold cache) by this run's edges and vertices per launch")
            roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                        "frac": achieved / hbm, "traffic": traffic, "traffic_note": note,
                        "bytes_model": model, "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})",
                        "launches": n, "avg_launch_us": ms * 1e3 / n, "alg_bytes_per_launch": alg / n,
                        "edges_per_launch": e_ / n,
                        "binding_roof": "L2 reductions (roofline_l2): the value arrays stay in L2"}
            if red_probe and hub_probe:
                roofline_l2 = {}
                peak = hub_probe[1]
                for k, (n, ms, e_, _, _, _) in kern.items():
                    rate = e_ / (ms * 1e-3) / 1e9
                    roofline_l2[k] = {"bound": "l2_reductions", "achieved": rate, "peak": peak,
                                      "unit": "G updates/s", "frac": rate / peak,
                                      "frac_of_uniform_probe": rate / red_probe[0]}
                roofline_l2["peak_source"] = ("hytg_probe_atomics_hub in this run: the R-MAT in-degree "
                                              "skew after hub sorting, with the kernels' per-SM replicas")
                roofline_l2["uniform_gops"] = red_probe[0]
                roofline_l2["skewed_gops"] = red_probe[1]
                roofline_l2["hub_skew_without_replicas_gops"] = hub_probe[0]
                # all PageRank reductions over its device time (kernels overlap on 5 streams)
                pr_e = sum(st["edges_relaxed"] + st["extra_edges"] for st in prs)
                pr_ms = sum(st["device_ms"] for st in prs)
                roofline_l2["pagerank_aggregate_gops"] = pr_e / (pr_ms * 1e-3) / 1e9
                roofline_l2["pagerank_aggregate_frac"] = pr_e / (pr_ms * 1e-3) / 1e9 / peak

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        smp = cpu_oracle_samples(g, s, algos)
        e_cpu = sum(v["edges"] for v in smp.values())
        s_cpu = sum(v["s"] for v in smp.values())
        cpu = {"value": e_cpu / s_cpu / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
               "sample": "oracle (single-threaded C) on the full graphs, once each: " +
                         ", ".join(v["what"] for v in smp.values()),
               "seconds": round(s_cpu, 2), "host_cores": os.cpu_count(),
               "per_algo": {a: {"cpu_gteps": v["gteps"], "gpu_gteps": per_algo[a]["gteps"],
                                "cpu_s": v["s"]} for a, v in smp.items()}}

    copy_gbs = [x for p in steps for a in algos if p[a]["tl"] for x in p[a]["tl"]["copy_gbs"]]
    h2d = sum(p[a]["h2d"] for p in steps for a in algos) // len(steps)
    d2h = sum(p[a]["d2h"] for p in steps for a in algos) // len(steps)
    link_per_step = link_bytes // len(steps)
    line = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 (PageRank f32)", "data": "synthetic",
        "config": dict(step_config(args, g, s, algos, world), graph_gen_s=round(t_gen, 1),
                       gteps_with_second_pass=(tot_edges + extra) / (max_ms * 1e-3) / 1e9,
                       per_algo_gteps={a: round(v["gteps"], 2) for a, v in per_algo.items()},
                       per_algo_ms={a: v["ms"] for a, v in per_algo.items()},
                       pagerank_l1_bound=per_algo.get("pagerank", {}).get("l1_bound"),
                       link_frac_of_probe=(link_bytes / (dev_ms * 1e-3) / 1e9 / probe)),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": "GTEPS", "h2d_bytes_per_step": h2d + link_per_step,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "roofline_l2": roofline_l2,
        "batched_vs_plain": batched,
        # Graph500-style BFS rate: each reached vertex's out-edges are relaxed
        # exactly once, so the BFS edge count is |E_reached|
        "graph500_bfs_gteps": (per_algo["bfs"]["gteps"] if "bfs" in per_algo else None),
        "host_link": {"achieved_gbs": link_bytes / (dev_ms * 1e-3) / 1e9,
                      "probe_before_gbs": probe_before[0] if probe_before else None,
                      "probe_after_gbs": probe_after[0] if probe_after else None,
                      "zerocopy_probe_gbs": probe_before[1] if probe_before else None,
                      "frac_of_probe": link_bytes / (dev_ms * 1e-3) / 1e9 / probe,
                      "bytes_per_step": link_per_step, "model_line_bytes_per_step": model_bytes // len(steps),
                      "f_copy_gbs_p10_p50_p90": [pct(copy_gbs, q) for q in (10, 50, 90)],
                      "while_transferring": per_route},
        "per_algo": per_algo,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    eng.close()
    eng_s.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
