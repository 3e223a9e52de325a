"""Autotuner for the engine's tunables (partition size, F-task merge width,
cost-model thresholds, streams), by coordinate descent over short runs.

Every trial is a real run through the C ABI; the objective is the device time
of the run (CUDA events, `device_ms`), averaged over `reps` runs after one
warm-up.  The tuner changes only parameters that leave results unchanged
(routes and partitioning never change what is computed), and restores the
best setting on the engine before returning.
"""
from __future__ import annotations

from typing import Dict, Iterable, List, Optional, Sequence

from . import hytg

DEFAULT_SPACE: Dict[str, List[float]] = {
    "part_bytes": [1 << 20, 2 << 20, 4 << 20, 8 << 20, 16 << 20],
    "k": [1, 2, 4, 8],
    "streams": [2, 4, 8],
    "MR": [16, 64, 256, 1024],
    "alpha": [0.6, 0.8, 1.0],
    "beta": [0.2, 0.4, 0.8],
}


def _measure(eng: "hytg.Engine", algo: str, sources, reps: int) -> float:
    a = hytg.ALGOS[algo]
    src = None if sources is None else list(sources)
    hytg.hytg_run(eng.ctx, a, src)
    total = 0.0
    for _ in range(reps):
        hytg.hytg_run(eng.ctx, a, src)
        total += eng.stats()["device_ms"]
    return total / reps


def autotune(eng: "hytg.Engine", workload: Sequence[tuple], space: Optional[Dict[str, Iterable[float]]] = None,
             reps: int = 2, rounds: int = 1, log=None) -> Dict[str, float]:
    """Tune `eng` for `workload`, a list of (algo, sources) pairs whose summed
    device time is minimised.  Returns the best parameters (also left set)."""
    space = {k: list(v) for k, v in (space or DEFAULT_SPACE).items()}
    best = {k: eng.get_param(k) for k in space}

    def cost() -> float:
        return sum(_measure(eng, algo, src, reps) for algo, src in workload)

    best_cost = cost()
    seen = {tuple(sorted(best.items())): best_cost}   # settings already measured
    if log:
        log(f"start {best} -> {best_cost:.2f} ms")
    for _ in range(rounds):
        for key, values in space.items():
            for v in values:
                trial = tuple(sorted(dict(best, **{key: v}).items()))
                if v == best[key] or trial in seen:
                    continue
                try:
                    eng.set_param(key, v)
                    c = cost()
                except hytg.HytgError:
                    eng.set_param(key, best[key])
                    continue
                seen[trial] = c
                if log:
                    log(f"  {key}={v} -> {c:.2f} ms")
                if c < best_cost:
                    best_cost, best[key] = c, v
            eng.set_param(key, best[key])
    if log:
        log(f"best {best} -> {best_cost:.2f} ms")
    return best
