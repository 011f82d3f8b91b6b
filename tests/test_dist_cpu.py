"""Multi-process host logic of bench.py on CPU: world size 2 over gloo.  Each
rank fixes its own lattice (replicas, no data-path collective); the step time
is the maximum over ranks and the throughput counts every rank's site updates."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.aggregate_over_ranks(1.5 + rank, 1000.0 * (rank + 1))
    out.put((rank, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2.5, 3000.0), (1, 2.5, 3000.0)]


def test_aggregate_single_process_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(0.7, 42.0) == (0.7, 42.0)
