"""Thin Python binding of the hytg C ABI (include/hytg.h).

Argument marshalling only: every step of the method runs in libhytg.so's
CUDA kernels.  The functions keep the C names; `Engine` is a small
convenience wrapper that owns one context.  There is no fallback: if the
library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhytg.so")

HYTG_OK, HYTG_ERR_ARG, HYTG_ERR_CUDA, HYTG_ERR_BUDGET = 0, 1, 2, 3
HYTG_ERR_HOSTMEM, HYTG_ERR_OVERFLOW, HYTG_ERR_TIMEOUT, HYTG_ERR_STATE = 4, 5, 6, 7
HYTG_BFS, HYTG_SSSP, HYTG_CC, HYTG_PAGERANK, HYTG_PPR = 0, 1, 2, 3, 4
ROUTE_NONE, ROUTE_CACHE, ROUTE_F, ROUTE_C, ROUTE_Z = 0, 1, 2, 3, 4
ROUTE_NAMES = ["none", "cache", "F", "C", "Z"]
UNREACHED = 0xFFFFFFFF
KERNEL_KINDS = ["init", "plan", "bin", "relax_cache", "relax_F", "gather_C", "relax_C", "relax_Z",
                "copy_F", "final", "cache_fill", "other"]
K_SECOND_PASS = 12                      # timeline kind of a second pass
ALGOS = {"bfs": HYTG_BFS, "sssp": HYTG_SSSP, "cc": HYTG_CC, "pagerank": HYTG_PAGERANK,
         "ppr": HYTG_PPR}

u64, u32, i32, dbl, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double, ctypes.c_void_p


class hytg_stats(ctypes.Structure):
    _fields_ = [("iterations", u32), ("status", u32), ("edges_relaxed", u64),
                ("vertices_processed", u64), ("route_partitions", u64 * 5),
                ("route_vertices", u64 * 5), ("route_edges", u64 * 5), ("link_bytes", u64 * 5),
                ("cache_fill_bytes", u64), ("f_tasks", u64), ("kernel_launches", u64),
                ("wall_ms", dbl), ("kernel_ms", dbl * 12), ("kernel_count", u64 * 12),
                ("pr_residual_sum", dbl), ("pr_rank_sum", dbl), ("device_ms", dbl),
                ("source_edges", u64), ("n_sources", u32), ("pad_", u32), ("extra_edges", u64),
                ("host_compact_ms", dbl), ("graph_launches", u64), ("graph_iterations", u64),
                ("second_pass_ms", dbl), ("second_pass_count", u64), ("second_pass_vertices", u64),
                ("route_busy_ms", dbl * 5), ("kernel_busy_ms", dbl * 13),
                ("link_sector_bytes", u64 * 5), ("link_line_bytes", u64 * 5),
                ("f_reused_tasks", u64), ("f_reused_bytes", u64),
                ("f_ahead_tasks", u64), ("f_ahead_hits", u64)]


class hytg_info(ctypes.Structure):
    _fields_ = [("V", u64), ("E", u64), ("weighted", u32), ("n_parts", u32), ("part_edges", u64),
                ("slot_edges", u64), ("n_slots", u32), ("n_cached", u32), ("budget_bytes", u64),
                ("budget_used_bytes", u64), ("compact_edges", u64), ("vertex_state_bytes", u64),
                ("pinned_host_bytes", u64)]


class hytg_iter_record(ctypes.Structure):
    _fields_ = [("active_vertices", u64), ("active_edges", u64), ("route_partitions", u32 * 5),
                ("f_tasks", u32), ("route_edges", u64 * 5), ("link_bytes", u64),
                ("device_ms", dbl)]


class hytg_timed_launch(ctypes.Structure):
    _fields_ = [("kind", u32), ("stream", u32), ("start_ms", dbl), ("end_ms", dbl), ("bytes", u64),
                ("edges", u64), ("vertices", u64), ("part_first", u32), ("part_last", u32)]


class hytg_serve_info(ctypes.Structure):
    _fields_ = [("frames", u32), ("frames_free", u32), ("slots_per_frame", u32), ("pad_", u32),
                ("frame_bytes", u64), ("edge_budget_bytes", u64), ("busy_slots", u64)]


class hytg_cost_params(ctypes.Structure):
    _fields_ = [("alpha", dbl), ("beta", dbl), ("gamma", dbl), ("m", u32), ("MR", u32)]


class HytgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"hytg status {status}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()


def load(path: Optional[str] = None):
    """Load libhytg.so (built by paper_2208_14935_gb300.build); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise HytgError(-1, f"{p} is missing: run `python -m paper_2208_14935_gb300.build`")
        lib = ctypes.CDLL(p)
        P = ctypes.POINTER
        sig = {
            "hytg_create": [P(vp), i32],
            "hytg_destroy": [vp],
            "hytg_load_csr": [vp, u64, u64, vp, vp, vp],
            "hytg_set_device_budget": [vp, u64],
            "hytg_set_param": [vp, ctypes.c_char_p, dbl],
            "hytg_get_param": [vp, ctypes.c_char_p, P(dbl)],
            "hytg_run": [vp, i32, vp, u32],
            "hytg_fetch_result": [vp, vp, u64],
            "hytg_fetch_pagerank_state": [vp, vp, vp, u64],
            "hytg_get_stats": [vp, P(hytg_stats)],
            "hytg_get_info": [vp, P(hytg_info)],
            "hytg_get_partitions": [vp, vp, u32, P(u32)],
            "hytg_plan": [vp, i32, vp, vp, vp, u32],
            "hytg_probe_link": [vp, u64, u32, P(dbl), P(dbl)],
            "hytg_get_iterations": [vp, vp, u32, P(u32)],
            "hytg_get_timeline": [vp, vp, u32, P(u32)],
            "hytg_hub_order": [u64, vp, vp, dbl, vp, P(u64)],
            "hytg_get_permutation": [vp, vp, u64],
            "hytg_probe_atomics": [vp, u64, u32, P(dbl), P(dbl)],
            "hytg_probe_atomics_hub": [vp, u64, u32, u32, P(dbl), P(dbl)],
            "hytg_probe_frame_push": [vp, u64, u32, u32, P(dbl)],
            "hytg_serve_begin": [vp, i32, u32],
            "hytg_serve_admit": [vp, u32, u32],
            "hytg_serve_step": [vp, P(u64), P(u64)],
            "hytg_serve_fetch": [vp, u32, vp, u64],
            "hytg_serve_end": [vp],
            "hytg_serve_get_info": [vp, P(hytg_serve_info)],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = i32
        lib.hytg_plan_noalloc.argtypes = [i32, vp, vp, u64, vp, u32, u32, P(hytg_cost_params), vp, vp, vp]
        lib.hytg_plan_noalloc.restype = i32
        lib.hytg_status_str.argtypes = [i32]
        lib.hytg_status_str.restype = ctypes.c_char_p
        lib.hytg_last_error.argtypes = [vp]
        lib.hytg_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(vp)


def _check(ctx, status: int):
    if status != HYTG_OK:
        lib = load()
        msg = lib.hytg_last_error(ctx).decode() if ctx else lib.hytg_status_str(status).decode()
        raise HytgError(status, msg or lib.hytg_status_str(status).decode())


# ------------------------------------------------------- C-named wrappers --
def hytg_create(device: int = 0):
    h = vp()
    _check(None, load().hytg_create(ctypes.byref(h), device))
    return h


def hytg_destroy(ctx):
    _check(None, load().hytg_destroy(ctx))


def hytg_load_csr(ctx, g):
    off = np.ascontiguousarray(g.off, np.uint64)
    dst = np.ascontiguousarray(g.dst, np.uint32)
    w = None if g.w is None else np.ascontiguousarray(g.w, np.uint32)
    _check(ctx, load().hytg_load_csr(ctx, g.V, g.E, _ptr(off), _ptr(dst), _ptr(w)))


def hytg_set_device_budget(ctx, nbytes: int):
    _check(ctx, load().hytg_set_device_budget(ctx, int(nbytes)))


def hytg_set_param(ctx, key: str, value: float):
    _check(ctx, load().hytg_set_param(ctx, key.encode(), float(value)))


def hytg_get_param(ctx, key: str) -> float:
    v = dbl()
    _check(ctx, load().hytg_get_param(ctx, key.encode(), ctypes.byref(v)))
    return v.value


def hytg_run(ctx, algo: int, sources: Optional[Sequence[int]] = None):
    src = None if sources is None else np.ascontiguousarray(sources, np.uint32)
    n = 0 if src is None else len(src)
    _check(ctx, load().hytg_run(ctx, int(algo), _ptr(src), n))


def hytg_fetch_result(ctx, V: int, algo: int, n_sources: int = 1) -> np.ndarray:
    dt = np.float32 if algo in (HYTG_PAGERANK, HYTG_PPR) else np.uint32
    out = np.empty(V * n_sources, dtype=dt)
    _check(ctx, load().hytg_fetch_result(ctx, _ptr(out), out.nbytes))
    return out if n_sources == 1 else out.reshape(n_sources, V)


def hytg_fetch_pagerank_state(ctx, V: int):
    rank = np.empty(V, np.float32)
    delta = np.empty(V, np.float32)
    _check(ctx, load().hytg_fetch_pagerank_state(ctx, _ptr(rank), _ptr(delta), V))
    return rank, delta


def hytg_get_stats(ctx) -> Dict:
    s = hytg_stats()
    _check(ctx, load().hytg_get_stats(ctx, ctypes.byref(s)))
    d = {}
    for name, _ in hytg_stats._fields_:
        v = getattr(s, name)
        d[name] = list(v) if hasattr(v, "__len__") else v
    return d


def hytg_get_info(ctx) -> Dict:
    s = hytg_info()
    _check(ctx, load().hytg_get_info(ctx, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in hytg_info._fields_}


def hytg_get_partitions(ctx) -> np.ndarray:
    n = u32()
    _check(ctx, load().hytg_get_partitions(ctx, None, 0, ctypes.byref(n)))
    vb = np.empty(n.value + 1, np.uint64)
    _check(ctx, load().hytg_get_partitions(ctx, _ptr(vb), n.value + 1, ctypes.byref(n)))
    return vb


def hytg_plan(ctx, algo: int, active: np.ndarray, n_parts: int):
    act = np.ascontiguousarray(active, np.uint8)
    routes = np.empty(n_parts, np.uint8)
    counts = np.empty(3 * n_parts, np.uint64)
    _check(ctx, load().hytg_plan(ctx, int(algo), _ptr(act), _ptr(routes), _ptr(counts), n_parts))
    return routes, counts.reshape(n_parts, 3)


def hytg_plan_noalloc(algo: int, frontier_ptr: int, offsets_ptr: int, V: int, vbounds_ptr: int,
                      n_parts: int, n_cached: int, routes_ptr: int, counts_ptr: int,
                      params: Optional[Dict[str, float]] = None, stream: int = 0) -> int:
    """Allocation-free planning on caller-owned device buffers (pointers as
    integers); returns the hytg_status without raising."""
    prm = None
    if params is not None:
        prm = hytg_cost_params(params.get("alpha", 0.8), params.get("beta", 0.4),
                               params.get("gamma", 0.625), int(params.get("m", 128)),
                               int(params.get("MR", 256)))
    return load().hytg_plan_noalloc(int(algo), vp(frontier_ptr), vp(offsets_ptr), V, vp(vbounds_ptr),
                                    n_parts, n_cached, None if prm is None else ctypes.byref(prm),
                                    vp(routes_ptr), vp(counts_ptr), vp(stream) if stream else None)


def hytg_hub_order(g, frac: float = 0.08):
    """Hub-sorting order (pure host): perm[n] = original id of internal vertex n."""
    off = np.ascontiguousarray(g.off, np.uint64)
    dst = np.ascontiguousarray(g.dst, np.uint32)
    perm = np.empty(g.V, np.uint32)
    nh = u64()
    _check(None, load().hytg_hub_order(g.V, _ptr(off), _ptr(dst), float(frac), _ptr(perm),
                                       ctypes.byref(nh)))
    return perm, nh.value


def hytg_get_permutation(ctx, V: int) -> np.ndarray:
    perm = np.empty(V, np.uint32)
    _check(ctx, load().hytg_get_permutation(ctx, _ptr(perm), V))
    return perm


def hytg_probe_link(ctx, nbytes: int = 1 << 30, reps: int = 10):
    a, b = dbl(), dbl()
    _check(ctx, load().hytg_probe_link(ctx, int(nbytes), reps, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def hytg_probe_atomics(ctx, n: int = 1 << 28, reps: int = 5):
    a, b = dbl(), dbl()
    _check(ctx, load().hytg_probe_atomics(ctx, int(n), reps, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def hytg_probe_atomics_hub(ctx, n: int = 1 << 28, reps: int = 5, n_rep: int = 4096):
    a, b = dbl(), dbl()
    _check(ctx, load().hytg_probe_atomics_hub(ctx, int(n), reps, n_rep, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def hytg_probe_frame_push(ctx, n: int = 1 << 26, reps: int = 3, width: int = 4) -> float:
    """1e9 pushes/s of a frame of 8 floats to random vertices, as 8 / width
    reductions of `width` floats."""
    a = dbl()
    _check(ctx, load().hytg_probe_frame_push(ctx, int(n), reps, width, ctypes.byref(a)))
    return a.value


def hytg_serve_begin(ctx, algo: int, n_slots: int):
    _check(ctx, load().hytg_serve_begin(ctx, int(algo), int(n_slots)))


def hytg_serve_admit(ctx, slot: int, source: int):
    _check(ctx, load().hytg_serve_admit(ctx, int(slot), int(source)))


def hytg_serve_step(ctx):
    fin, busy = u64(), u64()
    _check(ctx, load().hytg_serve_step(ctx, ctypes.byref(fin), ctypes.byref(busy)))
    return fin.value, busy.value


def hytg_serve_fetch(ctx, slot: int, V: int, algo: int) -> np.ndarray:
    out = np.empty(V, dtype=np.float32 if algo == HYTG_PPR else np.uint32)
    _check(ctx, load().hytg_serve_fetch(ctx, int(slot), _ptr(out), out.nbytes))
    return out


def hytg_serve_get_info(ctx) -> Dict:
    s = hytg_serve_info()
    _check(ctx, load().hytg_serve_get_info(ctx, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in hytg_serve_info._fields_ if name != "pad_"}


def hytg_serve_end(ctx):
    _check(ctx, load().hytg_serve_end(ctx))


def hytg_get_iterations(ctx):
    n = u32()
    _check(ctx, load().hytg_get_iterations(ctx, None, 0, ctypes.byref(n)))
    arr = (hytg_iter_record * max(1, n.value))()
    _check(ctx, load().hytg_get_iterations(ctx, arr, n.value, ctypes.byref(n)))
    out = []
    for r in arr[: n.value]:
        out.append({name: (list(getattr(r, name)) if hasattr(getattr(r, name), "__len__")
                           else getattr(r, name)) for name, _ in hytg_iter_record._fields_})
    return out


def hytg_get_timeline(ctx) -> np.ndarray:
    """The last run's timed launches as a numpy structured array (fields of
    hytg_timed_launch)."""
    n = u32()
    _check(ctx, load().hytg_get_timeline(ctx, None, 0, ctypes.byref(n)))
    arr = (hytg_timed_launch * max(1, n.value))()
    _check(ctx, load().hytg_get_timeline(ctx, arr, n.value, ctypes.byref(n)))
    dt = np.dtype([("kind", np.uint32), ("stream", np.uint32), ("start_ms", np.float64),
                   ("end_ms", np.float64), ("bytes", np.uint64), ("edges", np.uint64),
                   ("vertices", np.uint64), ("part_first", np.uint32), ("part_last", np.uint32)])
    assert dt.itemsize == ctypes.sizeof(hytg_timed_launch)
    return np.frombuffer(bytes(arr), dtype=dt, count=n.value).copy()


# ------------------------------------------------------------ convenience --
class Engine:
    """One hytg context with a loaded graph."""

    def __init__(self, g=None, budget: Optional[int] = None, device: int = 0,
                 params: Optional[Dict[str, float]] = None):
        self.ctx = hytg_create(device)
        self.V = 0
        for k, v in (params or {}).items():
            self.set_param(k, v)
        if g is not None:
            self.load(g)
        if budget is not None:
            self.set_budget(budget)

    def close(self):
        if self.ctx:
            hytg_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, g):
        hytg_load_csr(self.ctx, g)
        self.V = g.V

    def set_budget(self, nbytes: int):
        hytg_set_device_budget(self.ctx, nbytes)

    def set_param(self, key: str, value: float):
        hytg_set_param(self.ctx, key, value)

    def get_param(self, key: str) -> float:
        return hytg_get_param(self.ctx, key)

    def run(self, algo, source=None) -> np.ndarray:
        """source: None, one vertex id, or a sequence of ids (a batched run,
        whose result has one row per source)."""
        a = ALGOS[algo] if isinstance(algo, str) else int(algo)
        if source is None:
            hytg_run(self.ctx, a, None)
            return hytg_fetch_result(self.ctx, self.V, a)
        if np.ndim(source) == 0:
            hytg_run(self.ctx, a, [int(source)])
            return hytg_fetch_result(self.ctx, self.V, a)
        srcs = [int(x) for x in source]
        hytg_run(self.ctx, a, srcs)
        return hytg_fetch_result(self.ctx, self.V, a, len(srcs))

    def stats(self) -> Dict:
        return hytg_get_stats(self.ctx)

    def info(self) -> Dict:
        return hytg_get_info(self.ctx)

    def partitions(self) -> np.ndarray:
        return hytg_get_partitions(self.ctx)

    def plan(self, algo, active: np.ndarray):
        a = ALGOS[algo] if isinstance(algo, str) else int(algo)
        n = self.info()["n_parts"]
        return hytg_plan(self.ctx, a, active, n)

    def permutation(self) -> np.ndarray:
        return hytg_get_permutation(self.ctx, self.V)

    def timeline(self) -> np.ndarray:
        return hytg_get_timeline(self.ctx)

    def iterations(self):
        return hytg_get_iterations(self.ctx)

    def pagerank_state(self):
        return hytg_fetch_pagerank_state(self.ctx, self.V)

    def probe_link(self, nbytes: int = 1 << 30, reps: int = 10):
        return hytg_probe_link(self.ctx, nbytes, reps)

    def probe_atomics(self, n: int = 1 << 28, reps: int = 5):
        return hytg_probe_atomics(self.ctx, n, reps)
