"""Host logic of the autotuner (coordinate descent over engine parameters),
against a fake engine whose device time is a known function of the
parameters; no GPU."""
import pytest

from paper_2208_14935_gb300 import autotune as at
from paper_2208_14935_gb300 import hytg


class FakeEngine:
    """device_ms = sum of per-parameter costs; part_bytes 16 MiB is refused."""

    def __init__(self):
        self.ctx = object()
        self.p = {"part_bytes": 4 << 20, "k": 4, "MR": 256}
        self.runs = 0

    def get_param(self, k):
        return self.p[k]

    def set_param(self, k, v):
        if k == "part_bytes" and v == 16 << 20:
            raise hytg.HytgError(hytg.HYTG_ERR_ARG, "refused")
        self.p[k] = v

    def cost(self):
        c = {1 << 20: 5.0, 2 << 20: 3.0, 4 << 20: 4.0, 8 << 20: 6.0}[self.p["part_bytes"]]
        c += {1: 3.0, 2: 1.0, 4: 2.0, 8: 2.5}[self.p["k"]]
        c += {64: 1.0, 256: 2.0, 1024: 0.5}[self.p["MR"]]
        return c

    def stats(self):
        return {"device_ms": self.cost()}


@pytest.fixture
def fake(monkeypatch):
    eng = FakeEngine()

    def run(ctx, algo, src):
        eng.runs += 1

    monkeypatch.setattr(hytg, "hytg_run", run)
    return eng


def test_coordinate_descent_finds_the_separable_optimum(fake):
    space = {"part_bytes": [1 << 20, 2 << 20, 4 << 20, 8 << 20, 16 << 20], "k": [1, 2, 4, 8],
             "MR": [64, 256, 1024]}
    best = at.autotune(fake, [("bfs", [0])], space=space, reps=2)
    assert best == {"part_bytes": 2 << 20, "k": 2, "MR": 1024}
    assert fake.p == best                       # left set on the engine
    # one warm-up + reps runs per measured setting; each setting measured once
    # (the refused 16 MiB is never run)
    trials = 1 + sum(len(v) - 1 for v in space.values()) - 1
    assert fake.runs == trials * (1 + 2)


def test_refused_value_restores_the_parameter(fake):
    best = at.autotune(fake, [("bfs", [0])], space={"part_bytes": [16 << 20]}, reps=1)
    assert best == {"part_bytes": 4 << 20}
    assert fake.p["part_bytes"] == 4 << 20


def test_no_improvement_keeps_the_start(fake):
    fake.p = {"part_bytes": 2 << 20, "k": 2, "MR": 1024}
    best = at.autotune(fake, [("sssp", [1, 2])], space={"k": [4, 8], "MR": [64]}, reps=1)
    assert best == {"k": 2, "MR": 1024}
