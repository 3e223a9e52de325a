"""Seeded synthetic graph generators (inputs only; no step of the method)."""
from .graphgen import (  # noqa: F401
    CSR, rmat, mesh, chung_lu, symmetrize, random_graph, build, draw,
)
