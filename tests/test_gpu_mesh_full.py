"""Parity on the full-size high-diameter mesh: a 16384 x 16384 4-neighbour
grid (268,435,456 vertices, 1,073,676,288 directed grid edges) plus 0.1 %
local shortcuts within +-16 rows and columns, weights uniform in [1, 1000],
device budget 20 % of the graph bytes.  BFS and SSSP from the corner and CC
(the mesh is symmetric) are compared element by element with the oracle;
these runs have thousands of iterations with tiny frontiers."""
import numpy as np
import pytest

from gen import graphgen as gg
from oracle import oracle as orc

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

W = H = 16384


@pytest.fixture(scope="module")
def mesh():
    return gg.mesh(W, H, shortcut_frac=0.001, radius=16, seed=1, wmax=1000)


@pytest.fixture(scope="module")
def eng(mesh):
    from paper_2208_14935_gb300 import build, hytg
    build.build()
    g = mesh
    nbytes = g.E * 8 + (g.V + 1) * 8
    e = hytg.Engine(g, budget=int(0.2 * nbytes), params={"part_bytes": 4 * 1024 * 1024})
    yield e
    e.close()


def test_mesh_bfs(mesh, eng):
    lv = eng.run("bfs", 0)
    st = eng.stats()
    assert st["iterations"] > 1000
    want, _ = orc.bfs(mesh, 0)
    assert np.array_equal(lv, want)


def test_mesh_sssp(mesh, eng):
    d = eng.run("sssp", 0)
    want, _, ovf = orc.sssp(mesh, 0)
    assert not ovf
    assert np.array_equal(d, want)


def test_mesh_cc(mesh, eng):
    lab = eng.run("cc")
    assert np.array_equal(lab, orc.cc(mesh))
