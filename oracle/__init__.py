"""ORACLE -- test infrastructure only.

A plain CPU statement of what the hybrid-transfer graph engine computes:
textbook BFS / Dijkstra / union-find / FP64 power-iteration PageRank in C
(hytg_oracle.c), and the cost model of Sec. V in exact rationals
(planner.py).  Only the tests, the smoke check and the benchmark's CPU
baseline use it; the CUDA library shares no code with it.
"""
from . import oracle, planner  # noqa: F401
from .oracle import build, UNREACHED  # noqa: F401
