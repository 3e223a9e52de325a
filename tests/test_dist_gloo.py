"""The N > 1 bench path on CPU: two gloo ranks aggregate throughput as the
sum of units over the slowest rank's time (replicas, no data-path collective)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, l = bench.dist_env()
    assert (r, w, l) == (rank, world, rank)
    units, ms = bench.aggregate(1000.0 * (rank + 1), 10.0 + 5.0 * rank, world)
    bench.barrier(world)
    out.put((rank, units, ms))
    dist.destroy_process_group()


def test_two_rank_aggregate():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, units, ms in res:
        assert units == 3000.0 and ms == 15.0
