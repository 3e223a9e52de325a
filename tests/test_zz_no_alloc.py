"""The allocation-free planning entry point (hytg_plan_noalloc) against the
regular one (hytg_plan) on the same frontier, on two calls in a row.

hytg_plan_noalloc serves callers that cannot allocate device memory (during
stream capture, or under a framework that owns all device memory); its
scratch is a static device array shared by every call.  The device buffers
below belong to the test (allocated with torch), not to the entry point.
Routes and counts are integers, so they must match exactly.
"""
import numpy as np
import pytest

from gen import graphgen as gg

pytestmark = pytest.mark.gpu


def test_plan_noalloc_matches_plan():
    torch = pytest.importorskip("torch")
    from paper_2208_14935_gb300 import build, hytg
    build.build()
    hytg.load()
    g = gg.rmat(16, seed=1)
    params = dict(alpha=0.8, beta=0.4, gamma=0.625, MR=8)
    e = hytg.Engine(params={"part_bytes": 64 * 1024, "hub_frac": 0.0, **params})
    e.load(g)
    e.set_budget(g.E * 8 // 4)
    vb = e.partitions()
    n = len(vb) - 1
    dev = torch.device("cuda", 0)
    off_d = torch.from_numpy(g.off.view(np.int64)).to(dev)
    vb_d = torch.from_numpy(vb.view(np.int64)).to(dev)
    routes_d = torch.empty(n, dtype=torch.uint8, device=dev)
    counts_d = torch.empty(3 * n, dtype=torch.int64, device=dev)
    rng = np.random.default_rng(21)
    for call, (algo, dens) in enumerate([("bfs", 0.02), ("sssp", 0.3)]):
        act = (rng.random(g.V) < dens).astype(np.uint8)
        want_routes, want_counts = e.plan(algo, act)
        n_cached = e.info()["n_cached"]
        pad = np.zeros(-(-g.V // 32) * 32, np.uint8)
        pad[:g.V] = act
        words = np.packbits(pad, bitorder="little").view(np.uint32)
        fr_d = torch.from_numpy(words.view(np.int32).copy()).to(dev)
        routes_d.fill_(255)
        counts_d.fill_(-1)           # the call must clear what starts at zero
        torch.cuda.synchronize()
        st = hytg.hytg_plan_noalloc(hytg.ALGOS[algo], fr_d.data_ptr(), off_d.data_ptr(), g.V,
                                    vb_d.data_ptr(), n, n_cached, routes_d.data_ptr(),
                                    counts_d.data_ptr(), params=params, stream=0)
        assert st == hytg.HYTG_OK, f"call {call}: status {st}"
        torch.cuda.synchronize()
        got_routes = routes_d.cpu().numpy()
        got_counts = counts_d.cpu().numpy().view(np.uint64).reshape(n, 3)
        assert np.array_equal(got_routes, want_routes), f"call {call}: routes differ"
        assert np.array_equal(got_counts, want_counts), f"call {call}: counts differ"
        assert len(set(got_routes.tolist())) > 1
    # sizes beyond the static array are rejected before any launch
    st = hytg.hytg_plan_noalloc(hytg.HYTG_BFS, fr_d.data_ptr(), off_d.data_ptr(), g.V, vb_d.data_ptr(),
                                65536 + 1, 0,
                                routes_d.data_ptr(), counts_d.data_ptr())
    assert st == hytg.HYTG_ERR_ARG
    e.close()
