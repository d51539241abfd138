"""The multi-process path of bench.py on CPU: two gloo ranks, each with its own
time and count, give the slowest rank's time and the summed count."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, c = bench.reduce_ranks(1.5 + rank, 10 * (rank + 1), world)
    out.put((rank, t, c))
    dist.destroy_process_group()


def test_reduce_ranks_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 2.5, 30.0), (1, 2.5, 30.0)]


def test_reduce_ranks_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_ranks(3.0, 7, 1) == (3.0, 7)
