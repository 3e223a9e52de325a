"""Python side of the seeded graph generators.

The C part (graphgen.c, built into libgraphgen.so beside this file) makes the
large graphs; `random_graph` makes small irregular test graphs with numpy.
Both produce CSR with uint64 offsets, uint32 destinations and uint32 weights.
Nothing here computes any step of the hybrid transfer method: these are
inputs shared by the oracle checks, the GPU tests and the benchmark.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile libgraphgen.so with gcc (portable flags, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
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
            lib.gg_rmat.argtypes = [i32, u64, dbl, dbl, dbl, u64, u32, i32, vp, vp, vp]
            lib.gg_mesh.argtypes = [u64, u64, u64, i32, u64, u32, i32, vp, vp, vp,
                                    ctypes.POINTER(u64)]
            lib.gg_chung_lu.argtypes = [u64, u64, dbl, dbl, u64, u32, i32, vp, vp, vp]
            lib.gg_symmetrize.argtypes = [u64, vp, vp, i32, vp, vp]
            lib.gg_draw.argtypes = [u64, u64, u64]
            lib.gg_draw.restype = u64
            for f in (lib.gg_rmat, lib.gg_mesh, lib.gg_chung_lu, lib.gg_symmetrize):
                f.restype = i32
            _lib = lib
    return _lib


def _nthreads(n: Optional[int]) -> int:
    return n if n else max(1, os.cpu_count() or 1)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class CSR:
    """A directed graph in CSR form; `w` is None for unweighted graphs."""
    V: int
    E: int
    off: np.ndarray          # uint64 [V + 1]
    dst: np.ndarray          # uint32 [E]
    w: Optional[np.ndarray]  # uint32 [E] or None
    name: str = ""

    def degrees(self) -> np.ndarray:
        return np.diff(self.off).astype(np.uint64)


def draw(seed: int, stream: int, i: int) -> int:
    """One value of the counter-based generator (splitmix64 of seed, stream, i)."""
    return int(_load().gg_draw(seed, stream, i))


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, wmax: int = 64, weights: bool = True, nthreads: Optional[int] = None,
         pinned_alloc=None) -> CSR:
    """R-MAT graph with 2^scale vertices and edge_factor * 2^scale edges."""
    V = 1 << scale
    E = edge_factor * V
    alloc = pinned_alloc or (lambda n, dt: np.empty(n, dtype=dt))
    off = np.empty(V + 1, dtype=np.uint64)
    dst = alloc(E, np.uint32)
    w = alloc(E, np.uint32) if weights else None
    rc = _load().gg_rmat(scale, E, a, b, c, seed, wmax, _nthreads(nthreads), _ptr(off), _ptr(dst), _ptr(w))
    if rc != 0:
        raise RuntimeError(f"gg_rmat failed ({rc})")
    return CSR(V, E, off, dst, w, f"rmat{scale}")


def mesh(W: int, H: int, shortcut_frac: float = 0.001, radius: int = 16, seed: int = 1,
         wmax: int = 1000, weights: bool = True, nthreads: Optional[int] = None) -> CSR:
    """W x H 4-neighbour grid plus int(shortcut_frac * W * H) undirected local shortcuts."""
    V = W * H
    n_short = int(shortcut_frac * V)
    lib = _load()
    off = np.empty(V + 1, dtype=np.uint64)
    E = ctypes.c_uint64(0)
    rc = lib.gg_mesh(W, H, n_short, radius, seed, wmax, _nthreads(nthreads), _ptr(off), None, None,
                     ctypes.byref(E))
    if rc != 0:
        raise RuntimeError(f"gg_mesh failed ({rc})")
    dst = np.empty(E.value, dtype=np.uint32)
    w = np.empty(E.value, dtype=np.uint32) if weights else None
    rc = lib.gg_mesh(W, H, n_short, radius, seed, wmax, _nthreads(nthreads), _ptr(off), _ptr(dst),
                     _ptr(w), ctypes.byref(E))
    if rc != 0:
        raise RuntimeError(f"gg_mesh failed ({rc})")
    return CSR(V, int(E.value), off, dst, w, f"mesh{W}x{H}")


def chung_lu(V: int, E: int, beta: float = 2.1, i0: float = 1.0, seed: int = 1, wmax: int = 255,
             weights: bool = True, nthreads: Optional[int] = None) -> CSR:
    off = np.empty(V + 1, dtype=np.uint64)
    dst = np.empty(E, dtype=np.uint32)
    w = np.empty(E, dtype=np.uint32) if weights else None
    rc = _load().gg_chung_lu(V, E, beta, i0, seed, wmax, _nthreads(nthreads), _ptr(off), _ptr(dst), _ptr(w))
    if rc != 0:
        raise RuntimeError(f"gg_chung_lu failed ({rc})")
    return CSR(V, E, off, dst, w, f"chunglu{V}")


def symmetrize(g: CSR, nthreads: Optional[int] = None) -> CSR:
    """Every edge u->v plus its reverse v->u (2E edges, unweighted)."""
    off2 = np.empty(g.V + 1, dtype=np.uint64)
    dst2 = np.empty(2 * g.E, dtype=np.uint32)
    rc = _load().gg_symmetrize(g.V, _ptr(g.off), _ptr(g.dst), _nthreads(nthreads), _ptr(off2), _ptr(dst2))
    if rc != 0:
        raise RuntimeError(f"gg_symmetrize failed ({rc})")
    return CSR(g.V, 2 * g.E, off2, dst2, None, g.name + "_sym")


def random_graph(V: int, E: int, seed: int, wmax: int = 64, skew: float = 0.0,
                 self_loops: bool = True, weights: bool = True) -> CSR:
    """Small irregular directed multigraph for tests (numpy, seeded).

    skew > 0 concentrates sources on low ids (a few high-degree vertices and
    many low-degree ones, like the power-law graphs of the paper's Sec. III).
    """
    rng = np.random.default_rng(seed)
    if V == 0:
        return CSR(0, 0, np.zeros(1, np.uint64), np.zeros(0, np.uint32),
                   np.zeros(0, np.uint32) if weights else None, "empty")
    if skew > 0:
        src = np.minimum((rng.pareto(skew, E) * V / 8).astype(np.int64), V - 1)
    else:
        src = rng.integers(0, V, E)
    dst = rng.integers(0, V, E)
    if not self_loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    w = rng.integers(1, wmax + 1, len(src)).astype(np.uint32)
    order = np.lexsort((w, dst, src))
    src, dst, w = src[order], dst[order], w[order]
    off = np.zeros(V + 1, dtype=np.uint64)
    np.add.at(off, src + 1, 1)
    off = np.cumsum(off).astype(np.uint64)
    return CSR(V, len(dst), off, dst.astype(np.uint32), w if weights else None, f"rand{V}_{seed}")
