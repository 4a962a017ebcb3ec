"""The multi-rank path of the bench on CPU: two gloo ranks (replicas) reduce
their timings to the slowest rank and sum their particle-steps."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 150.0][rank]                  # rank 1 is the slow one
    psteps = [4.0e9, 3.0e9][rank]
    t, v = bench.aggregate(ms, psteps, dist, "cpu")
    out[rank] = (t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        t, v = out[r]
        assert t == 150.0
        assert v == pytest.approx(7.0e9 / 0.150)


def test_single_rank_aggregation():
    sys.path.insert(0, ROOT)
    import bench
    t, v = bench.aggregate(200.0, 1.0e9)
    assert t == 200.0 and v == pytest.approx(5.0e9)
