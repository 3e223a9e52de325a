"""Benchmark: GTEPS of the hybrid-transfer engine at a capped device budget.

Workload (one "step"): on an R-MAT scale-24 graph (16,777,216 vertices,
268,435,456 directed edges, a=0.57 b=0.19 c=0.19 d=0.05, seed 1, uint32
weights uniform in [1, 64]) whose edge arrays live in pinned host memory,
with a device budget of 25 % of the graph bytes: BFS and SSSP from vertex 0,
connected components on the symmetrised graph (536,870,912 edges) and
delta-PageRank (damping 0.85, FP32 residual threshold 1e-9), each to
convergence through the C ABI.

value  = edges relaxed (sum over iterations of active out-edges, plus the
         second-pass relaxations over resident partitions, Sec. VI-A) / device
         time of the runs (CUDA events on the library's main stream, which
         joins all of its streams), summed over the K timed steps, over all
         ranks, divided by the slowest rank's time;
e2e    = the same edges over host wall time of hytg_run + hytg_fetch_result
         (the public calls), including the result copies to host memory.

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
    time, on the same engine, graph and budget.  Rate = per-source edges
    relaxed / device time (CUDA events), i.e. the throughput a user of many
    single-source queries gets."""
    rng = np.random.default_rng(7)
    cand = np.flatnonzero(np.diff(g.off.astype(np.int64)) > 0)
    out = {}
    for algo, k, n_plain in (("bfs", 64, 64), ("sssp", 64, n_plain_sssp), ("ppr", 32, n_plain_ppr)):
        src = rng.choice(cand, k, replace=False).tolist()
        a = hytg.ALGOS[algo]
        hytg.hytg_run(eng.ctx, a, src)                       # warm-up
        b_ms, b_edges = 0.0, 0
        for _ in range(2):
            hytg.hytg_run(eng.ctx, a, src)
            st = eng.stats()
            b_ms += st["device_ms"]
            b_edges += st["source_edges"]
        p_ms, p_edges = 0.0, 0
        for v in src[:n_plain]:
            hytg.hytg_run(eng.ctx, a, [v])
            st = eng.stats()
            p_ms += st["device_ms"]
            p_edges += st["edges_relaxed"]
        bg = b_edges / (b_ms * 1e-3) / 1e9
        pg = p_edges / (p_ms * 1e-3) / 1e9
        out[algo] = {"sources": k, "batched_gteps": bg, "batched_ms": b_ms / 2,
                     "plain_gteps": pg, "plain_ms_per_source": p_ms / n_plain,
                     "plain_sources_timed": n_plain, "speedup": bg / pg if pg else None}
    return out


# ------------------------------------------------------- reference arm ----
def cpu_oracle_sample(g, budget_s: float = 20.0):
    """The oracle (plain single-threaded C) on a bounded sample: BFS from 0,
    then Dijkstra from 0 if the BFS left time in the budget."""
    from oracle import oracle as orc
    t0 = time.perf_counter()
    _, e_bfs = orc.bfs(g, 0)
    t1 = time.perf_counter()
    edges, secs, sample = e_bfs, t1 - t0, "oracle BFS from vertex 0 on the full graph"
    if (t1 - t0) * 6 < budget_s:
        _, e_sp, _ = orc.sssp(g, 0)
        t2 = time.perf_counter()
        edges += e_sp
        secs = t2 - t0
        sample += " + oracle Dijkstra from vertex 0 on the full graph"
    return edges, secs, sample


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
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    g, s = make_graphs(args.scale)
    from oracle import oracle as orc
    orc.build()
    total_e, total_s = 0, 0.0
    sample = ""
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        lv, e = orc.bfs(g, 0)
        dt = time.perf_counter() - t0
        sample = "oracle FIFO BFS from vertex 0 on the full graph, one per step"
        if i >= args.warmup:
            total_e += e
            total_s += dt
    v = total_e / total_s / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": step_config(args, g, s, [a for a in args.algos.split(",") if a], 1),
            "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": sample},
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

    def one_step(collect):
        per = {}
        for algo in algos:
            e = eng_s if algo == "cc" else eng
            src = 0 if algo in ("bfs", "sssp") else None
            t0 = time.perf_counter()
            hytg.hytg_run(e.ctx, hytg.ALGOS[algo], None if src is None else [src])
            out = hytg.hytg_fetch_result(e.ctx, e.V, hytg.ALGOS[algo])
            wall = (time.perf_counter() - t0) * 1e3
            st = e.stats()
            per[algo] = {"stats": st, "wall_ms": wall, "d2h": out.nbytes,
                         "h2d": 0 if src is None else 4}
        return per

    for _ in range(args.warmup):
        one_step(False)
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    steps = []
    for _ in range(args.steps):
        steps.append(one_step(True))
    barrier(world)
    clk = clocks.stop()
    batched = None if args.no_batched else batched_vs_plain(hytg, eng, g)
    red_probe = None if args.no_probe else eng.probe_atomics(1 << 28, 5)
    # the link probe runs after the timed region (it pins and frees 1 GiB)
    memcpy_gbs, zc_gbs = (float("nan"), float("nan")) if args.no_probe else eng.probe_link(1 << 30, 10)

    # every relaxation of an active vertex's out-edges: planned iterations plus
    # the second passes over resident partitions (Sec. VI-A, on for PageRank)
    edges = sum(p[a]["stats"]["edges_relaxed"] + p[a]["stats"]["extra_edges"] for p in steps for a in algos)
    dev_ms = sum(p[a]["stats"]["device_ms"] for p in steps for a in algos)
    wall_ms = sum(p[a]["wall_ms"] for p in steps for a in algos)
    launches = sum(p[a]["stats"]["kernel_launches"] for p in steps for a in algos)
    tot_edges, max_ms = aggregate(float(edges), dev_ms, world)
    tot_edges_w, max_wall = aggregate(float(edges), wall_ms, world)
    value = tot_edges / (max_ms * 1e-3) / 1e9
    e2e = tot_edges_w / (max_wall * 1e-3) / 1e9

    # host link: bytes moved over the link by the F, C and Z routes / device time
    link_bytes = sum(sum(p[a]["stats"]["link_bytes"]) for p in steps for a in algos)
    link_gbs = link_bytes / (dev_ms * 1e-3) / 1e9
    # per route: its bytes over the time its transfers were in flight (union
    # over streams of the F copies / C gathers / Z relaxes, timing on)
    per_route = {}
    for r, name in ((2, "F"), (3, "C"), (4, "Z")):
        b = sum(p[a]["stats"]["link_bytes"][r] for p in steps for a in algos)
        busy = sum(p[a]["stats"]["route_busy_ms"][r] for p in steps for a in algos)
        per_route[name] = {"bytes": b, "busy_ms": round(busy, 2),
                           "gbs": b / (busy * 1e-3) / 1e9 if busy > 0 else None}
    per_algo = {}
    for a in algos:
        ed = sum(p[a]["stats"]["edges_relaxed"] + p[a]["stats"]["extra_edges"] for p in steps)
        ms = sum(p[a]["stats"]["device_ms"] for p in steps)
        st = steps[-1][a]["stats"]
        kk = [sum(p[a]["stats"]["kernel_ms"][i] for p in steps) / len(steps) for i in range(12)]
        per_algo[a] = {"gteps": ed / (ms * 1e-3) / 1e9, "ms": ms / len(steps),
                       "ms_each_step": [round(p[a]["stats"]["device_ms"], 2) for p in steps],
                       "kernel_ms": {hytg.KERNEL_KINDS[i]: round(kk[i], 2) for i in range(12) if kk[i]},
                       "iterations": st["iterations"], "edges_relaxed": st["edges_relaxed"],
                       "second_pass_edges": st["extra_edges"],
                       "second_pass_ms": round(sum(p[a]["stats"]["second_pass_ms"] for p in steps) / len(steps), 2),
                       "graph_iterations": st["graph_iterations"],
                       "route_partitions": dict(zip(hytg.ROUTE_NAMES, st["route_partitions"])),
                       "route_edges": dict(zip(hytg.ROUTE_NAMES, st["route_edges"])),
                       "link_bytes": sum(st["link_bytes"])}

    # dominant kernel kind over the timed steps (per-kind CUDA events)
    kinds = hytg.KERNEL_KINDS
    kms = [0.0] * 12
    kcnt = [0] * 12
    for p in steps:
        for a in algos:
            for i in range(12):
                kms[i] += p[a]["stats"]["kernel_ms"][i]
                kcnt[i] += p[a]["stats"]["kernel_count"][i]
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    roofline, roofline_l2, roofline_relax = None, None, None
    if not args.no_timing and "pagerank" in algos:
        # PageRank is most of the step.  Its two heaviest kernels in the ncu
        # launch list (profiles/) are the second pass over resident partitions
        # (k_second_pass<PageRank>, ~50-60 %) and the F-route relax
        # (k_relax<PageRank>, ~20-30 %); `roofline` is whichever took longer
        # in this run, the other is reported beside it.
        pr = [p["pagerank"]["stats"] for p in steps]
        ms_f = sum(st["kernel_ms"][4] for st in pr)
        n_f = sum(st["kernel_count"][4] for st in pr)
        e_f = sum(st["route_edges"][2] for st in pr)
        v_f = sum(st["route_vertices"][2] for st in pr)
        busy_f = sum(st["kernel_busy_ms"][4] for st in pr)
        busy_sp = sum(st["kernel_busy_ms"][12] for st in pr)
        ms_sp = sum(st["second_pass_ms"] for st in pr)
        n_sp = sum(st["second_pass_count"] for st in pr)
        e_sp = sum(st["extra_edges"] for st in pr)
        v_sp = sum(st["second_pass_vertices"] for st in pr)
        if ms_f > 0 and n_f > 0:
            # algorithmic bytes: 4 B edge + 8 B value read-modify-write per edge,
            # 20 B list entry per active vertex
            alg = e_f * 12 + v_f * 20
            achieved = alg / (ms_f * 1e-3) / 1e9
            # DRAM bytes per launch from the ncu capture of the same kernel on an
            # F task of the same size (profiles/k_relax_pagerank_rmat22.md):
            # 30.8 MB for 4.37 M edges, scaled by this run's edges per launch
            traffic = 30.8e6 / 4.37e6 * (e_f / n_f)
            roofline_relax = {"kernel": "k_relax<PageRank> F route", "bound": "hbm", "achieved": achieved,
                              "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                              "bytes_model": "per edge 4 + 8 (value RMW), per active vertex 20",
                              "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})",
                              "launches": n_f, "avg_launch_us": ms_f * 1e3 / n_f,
                              "alg_bytes_per_launch": alg / n_f,
                              # the same bytes over the wall time during which any F
                              # relax was running (launches overlap on 4 streams)
                              "achieved_while_running": alg / (busy_f * 1e-3) / 1e9 if busy_f else None}
        if ms_sp > 0 and n_sp > 0:
            # per edge 4 B edge + 8 B value RMW; per scanned vertex 16 B offsets,
            # 4 B delta read, 8 B delta and rank reductions
            alg = e_sp * 12 + v_sp * 28
            achieved = alg / (ms_sp * 1e-3) / 1e9
            rl_sp = {"kernel": "k_second_pass<PageRank>", "bound": "hbm", "achieved": achieved,
                     "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                     "traffic_note": "not captured for a launch of known size; a cold-cache capture of "
                                     "one R-MAT 22 launch read 55.5 MB (profiles/)",
                     "bytes_model": "per edge 4 + 8 (value RMW), per scanned vertex 28",
                     "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})",
                     "launches": n_sp, "avg_launch_us": ms_sp * 1e3 / n_sp,
                     "alg_bytes_per_launch": alg / n_sp,
                     "achieved_while_running": alg / (busy_sp * 1e-3) / 1e9 if busy_sp else None}
            if roofline_relax is None or ms_sp > ms_f:
                roofline, roofline_relax = rl_sp, roofline_relax
            else:
                roofline, roofline_relax = roofline_relax, rl_sp
        else:
            roofline, roofline_relax = roofline_relax, None
        if red_probe and ms_f > 0:
            rate = e_f / (ms_f * 1e-3) / 1e9
            roofline_l2 = {"kernel": "k_relax<PageRank> F route", "bound": "l2_reductions",
                           "achieved": rate, "peak": red_probe[0], "unit": "G updates/s",
                           "frac": rate / red_probe[0],
                           "achieved_while_running": e_f / (busy_f * 1e-3) / 1e9 if busy_f else None,
                           "peak_source": "hytg_probe_atomics, uniform targets, same run",
                           "skewed_targets_gops": red_probe[1]}
    elif not args.no_timing:
        relax = {"relax_Z": 7, "relax_cache": 3, "relax_F": 4, "relax_C": 6, "gather_C": 5}
        dom = max(relax, key=lambda k: kms[relax[k]])
        route_of = {"relax_Z": 4, "relax_cache": 1, "relax_F": 2, "relax_C": 3, "gather_C": 3}
        r = route_of[dom]
        alg_bytes = 0
        for p in steps:
            for a in algos:
                d1 = 8 if a == "sssp" else 4
                st = p[a]["stats"]
                alg_bytes += st["route_edges"][r] * (d1 + 8) + st["route_vertices"][r] * 20
        ms = kms[relax[dom]]
        achieved = alg_bytes / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "traffic": None,
                    "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        e_cpu, s_cpu, sample = cpu_oracle_sample(g)
        cpu = {"value": e_cpu / s_cpu / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
               "sample": sample, "seconds": s_cpu, "host_cores": os.cpu_count()}

    h2d = sum(p[a]["h2d"] for p in steps for a in algos) // len(steps)
    d2h = sum(p[a]["d2h"] for p in steps for a in algos) // len(steps)
    link_per_step = link_bytes // len(steps)
    line = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 (PageRank f32)", "data": "synthetic",
        "config": dict(step_config(args, g, s, algos, world), graph_gen_s=round(t_gen, 1)),
        "host_link": {"achieved_gbs": link_gbs, "memcpy_probe_gbs": memcpy_gbs,
                      "zerocopy_probe_gbs": zc_gbs, "frac_of_measured": link_gbs / memcpy_gbs,
                      "bytes_per_step": link_per_step,
                      "while_transferring": {k: dict(v, frac_of_measured=(v["gbs"] / memcpy_gbs
                                                                         if v["gbs"] else None))
                                             for k, v in per_route.items()}},
        "batched_vs_plain": batched,
        "roofline": roofline,
        "roofline_l2": roofline_l2,
        "roofline_other": roofline_relax,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": "GTEPS", "h2d_bytes_per_step": h2d + link_per_step,
                "d2h_bytes_per_step": d2h},
        # Graph500-style BFS rate: each reached vertex's out-edges are relaxed
        # exactly once, so the BFS edge count is |E_reached|
        "graph500_bfs_gteps": (per_algo["bfs"]["gteps"] if "bfs" in per_algo else None),
        "gpu_launches": launches,
        "clocks": clk,
        "per_algo": per_algo,
        "kernel_ms": {kinds[i]: kms[i] for i in range(12) if kcnt[i]},
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
