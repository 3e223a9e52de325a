"""GB300 hybrid-transfer graph engine (HyTGraph's HyTM method, arXiv 2208.14935).

The compute path is libhytg.so (hand-written CUDA for sm_103a behind the C ABI
of include/hytg.h); `hytg` is its thin ctypes binding.
"""
from . import hytg  # noqa: F401
from .hytg import Engine, HytgError  # noqa: F401
