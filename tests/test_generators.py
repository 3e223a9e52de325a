"""Seeded generators: exact sizes, determinism for any thread count, shape."""
import numpy as np

from gen import graphgen as gg
from oracle import oracle as orc


def test_rmat_exact_and_deterministic():
    a = gg.rmat(14, nthreads=1)
    b = gg.rmat(14, nthreads=5)
    assert a.V == 1 << 14 and a.E == 16 << 14 and int(a.off[-1]) == a.E
    assert np.array_equal(a.off, b.off) and np.array_equal(a.dst, b.dst) and np.array_equal(a.w, b.w)
    assert a.w.min() >= 1 and a.w.max() <= 64
    deg = a.degrees()
    # a = 0.57 > d: vertex 0 is the largest hub, and many vertices have no out-edge
    assert int(np.argmax(deg)) == 0
    assert (deg == 0).mean() > 0.2
    # rows sorted by (dst, w)
    for v in range(0, a.V, 997):
        row = a.dst[a.off[v]:a.off[v + 1]]
        assert np.all(np.diff(row.astype(np.int64)) >= 0)
    c = gg.rmat(14, seed=2)
    assert not np.array_equal(a.dst, c.dst)


def test_mesh_shape():
    W, H = 40, 25
    m = gg.mesh(W, H, shortcut_frac=0.01, radius=4)
    assert m.V == W * H
    grid_edges = 2 * (W * (H - 1) + H * (W - 1))
    n_short = int(0.01 * W * H)
    assert m.E == grid_edges + 2 * n_short
    assert orc.is_symmetric(m)
    deg = m.degrees().astype(np.int64)
    base = np.array([(r > 0) + (c > 0) + (c < W - 1) + (r < H - 1) for r in range(H) for c in range(W)])
    extra = deg - base
    assert extra.min() >= 0 and extra.sum() == 2 * n_short
    assert m.w.min() >= 1 and m.w.max() <= 1000
    # shortcuts stay within +-radius rows and columns
    for u in range(m.V):
        for v in m.dst[m.off[u]:m.off[u + 1]]:
            assert abs(int(v) // W - u // W) <= 4 and abs(int(v) % W - u % W) <= 4
    m2 = gg.mesh(W, H, shortcut_frac=0.01, radius=4, nthreads=1)
    assert np.array_equal(m.dst, m2.dst) and np.array_equal(m.w, m2.w)


def test_symmetrize():
    g = gg.random_graph(300, 2000, seed=3)
    s = gg.symmetrize(g)
    assert s.E == 2 * g.E and orc.is_symmetric(s)


def test_chung_lu_shape():
    g = gg.chung_lu(1 << 14, 1 << 18, beta=2.1)
    deg = g.degrees()
    assert int(g.off[-1]) == 1 << 18
    assert deg[:16].mean() > 20 * deg.mean()      # power-law head
    assert np.array_equal(g.dst, gg.chung_lu(1 << 14, 1 << 18, beta=2.1, nthreads=1).dst)
