"""ORACLE -- test infrastructure only (never imported by the product path).

ctypes wrappers over hytg_oracle.c (plain single-threaded C, built into
liboracle.so beside this file) plus small numpy helpers.  Only the tests,
`__graft_entry__.smoke()` and the benchmark's CPU-baseline / reference leg
call into this package.

Every function states the passage of the paper whose result it computes:
the method (hybrid transfer management, Sec. IV-VI) reaches exactly the
results of the plain algorithms named in Sec. VII-A, so these are the plain
definitions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

UNREACHED = 0xFFFFFFFF
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hytg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C, -O2, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u64, u32, i32, dbl, vp = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_void_p)
            sig = {
                "or_bfs": [u64, vp, vp, u32, vp, vp],
                "or_sssp_dijkstra": [u64, vp, vp, vp, u32, vp, vp],
                "or_sssp_bellman_ford": [u64, vp, vp, vp, u32, vp],
                "or_cc_unionfind": [u64, vp, vp, vp],
                "or_cc_bfs": [u64, vp, vp, vp],
                "or_is_symmetric": [u64, vp, vp],
                "or_pagerank": [u64, vp, vp, dbl, dbl, i32, u32, vp, vp, vp],
                "or_pagerank_residual": [u64, vp, vp, dbl, u32, vp, vp],
                "or_bfs_certify": [u64, vp, vp, u32, vp, vp],
                "or_sssp_certify": [u64, vp, vp, vp, u32, vp, vp],
                "or_cc_certify": [u64, vp, vp, vp, u64, vp],
                "or_partition_counts": [u64, vp, vp, u32, vp, u32, u32, u32, vp, vp, vp],
            }
            for name, args in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = i32
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ------------------------------------------------------------ algorithms --
def bfs(g, src: int) -> Tuple[np.ndarray, int]:
    """Hop levels from `src` (Sec. VII-A BFS); returns (level, edges scanned)."""
    off, dst = _c(g.off, np.uint64), _c(g.dst, np.uint32)
    level = np.empty(g.V, np.uint32)
    scanned = ctypes.c_uint64(0)
    rc = _load().or_bfs(g.V, _p(off), _p(dst), src, _p(level), ctypes.byref(scanned))
    if rc != 0:
        raise ValueError(f"or_bfs rc={rc}")
    return level, int(scanned.value)


def sssp(g, src: int) -> Tuple[np.ndarray, int, bool]:
    """Dijkstra distances (Sec. II-A, Fig. 1 SSSP); returns (dist, edges scanned, overflow)."""
    off, dst, w = _c(g.off, np.uint64), _c(g.dst, np.uint32), _c(g.w, np.uint32)
    dist = np.empty(g.V, np.uint32)
    scanned = ctypes.c_uint64(0)
    rc = _load().or_sssp_dijkstra(g.V, _p(off), _p(dst), _p(w), src, _p(dist), ctypes.byref(scanned))
    if rc < 0:
        raise ValueError(f"or_sssp_dijkstra rc={rc}")
    return dist, int(scanned.value), rc == 1


def sssp_bellman_ford(g, src: int, unit_weights: bool = False) -> np.ndarray:
    """Alternate SSSP (and, with unit weights, an alternate BFS)."""
    off, dst = _c(g.off, np.uint64), _c(g.dst, np.uint32)
    w = None if unit_weights else _c(g.w, np.uint32)
    dist = np.empty(g.V, np.uint32)
    rc = _load().or_sssp_bellman_ford(g.V, _p(off), _p(dst), _p(w), src, _p(dist))
    if rc < 0:
        raise ValueError(f"or_sssp_bellman_ford rc={rc}")
    return dist


def cc(g) -> np.ndarray:
    """Weakly connected components by union-find, label = smallest id (Sec. VII-A CC)."""
    off, dst = _c(g.off, np.uint64), _c(g.dst, np.uint32)
    label = np.empty(g.V, np.uint32)
    _load().or_cc_unionfind(g.V, _p(off), _p(dst), _p(label))
    return label


def cc_bfs(g) -> np.ndarray:
    """Alternate CC for symmetric graphs (BFS from each unlabelled id, upwards)."""
    off, dst = _c(g.off, np.uint64), _c(g.dst, np.uint32)
    label = np.empty(g.V, np.uint32)
    _load().or_cc_bfs(g.V, _p(off), _p(dst), _p(label))
    return label


def is_symmetric(g) -> bool:
    off, dst = _c(g.off, np.uint64), _c(g.dst, np.uint32)
    return _load().or_is_symmetric(g.V, _p(off), _p(dst)) == 1


def pagerank(g, d: float = 0.85, tol: float = 1e-13, maxit: int = 1000,
             seed: Optional[int] = None) -> Tuple[np.ndarray, float, int]:
    """FP64 power iteration of x = (1-d) t + d A^T D_o^-1 x (Sec. VI-A delta
    PageRank's fixed point); t = 1 (PageRank) or e_seed (personalised).
    Returns (x normalised to sum 1, raw sum of the fixed point, iterations)."""
    off, dst = _c(g.off, np.uint64), _c(g.dst, np.uint32)
    x = np.empty(g.V, np.float64)
    raw = ctypes.c_double(0)
    it = ctypes.c_int(0)
    s = UNREACHED if seed is None else seed
    rc = _load().or_pagerank(g.V, _p(off), _p(dst), d, tol, maxit, s, _p(x), ctypes.byref(raw),
                             ctypes.byref(it))
    if rc != 0:
        raise ValueError(f"or_pagerank rc={rc}")
    return x, raw.value, it.value


def pagerank_residual(g, r: np.ndarray, d: float = 0.85, seed: Optional[int] = None) -> float:
    """|| (1-d) t + d A^T D_o^-1 r - r ||_1 on the unnormalised scale."""
    off, dst = _c(g.off, np.uint64), _c(g.dst, np.uint32)
    rr = _c(r, np.float64)
    res = ctypes.c_double(0)
    s = UNREACHED if seed is None else seed
    _load().or_pagerank_residual(g.V, _p(off), _p(dst), d, s, _p(rr), ctypes.byref(res))
    return res.value


# ---------------------------------------------------------- certificates --
def bfs_certify(g, src: int, level: np.ndarray) -> Tuple[int, int]:
    off, dst, lv = _c(g.off, np.uint64), _c(g.dst, np.uint32), _c(level, np.uint32)
    bad = ctypes.c_uint64(0)
    rc = _load().or_bfs_certify(g.V, _p(off), _p(dst), src, _p(lv), ctypes.byref(bad))
    return rc, int(bad.value)


def sssp_certify(g, src: int, dist: np.ndarray) -> Tuple[int, int]:
    off, dst, w, dd = _c(g.off, np.uint64), _c(g.dst, np.uint32), _c(g.w, np.uint32), _c(dist, np.uint32)
    bad = ctypes.c_uint64(0)
    rc = _load().or_sssp_certify(g.V, _p(off), _p(dst), _p(w), src, _p(dd), ctypes.byref(bad))
    return rc, int(bad.value)


def cc_certify(g, label: np.ndarray, n_components: int) -> Tuple[int, int]:
    off, dst, lb = _c(g.off, np.uint64), _c(g.dst, np.uint32), _c(label, np.uint32)
    bad = ctypes.c_uint64(0)
    rc = _load().or_cc_certify(g.V, _p(off), _p(dst), _p(lb), n_components, ctypes.byref(bad))
    return rc, int(bad.value)


# ------------------------------------------------- cost-model counting ----
def partition_counts(g, active: np.ndarray, vbounds, elem_bytes: int = 4, n_arrays: int = 1,
                     m: int = 128):
    """Per partition (Sec. V-A): |A_i|, sum of D_o over A_i, and the number of
    m-byte lines the active edge lists span (footnote to Eq. 3)."""
    off = _c(g.off, np.uint64)
    act = _c(active, np.uint8)
    vb = _c(vbounds, np.uint64)
    n = len(vb) - 1
    na, ae, ln = (np.zeros(n, np.uint64) for _ in range(3))
    _load().or_partition_counts(g.V, _p(off), _p(act), n, _p(vb), elem_bytes, n_arrays, m,
                                _p(na), _p(ae), _p(ln))
    return na, ae, ln
