"""Multi-rank path of bench.py on CPU: two gloo ranks (replicas of the whole
step, no data-path collective) agree on the slowest rank's time and report
the whole-job seconds per iteration over the steps of both ranks."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, v = bench.job_seconds_per_iter(1.0 + rank, steps=5, dist=dist)
    out[rank] = (t, v)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks(world):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        t, v = res[r]
        assert t == float(world)                     # slowest rank: 1.0 + (world - 1)
        assert v == pytest.approx(world / (5 * world))


def test_single_rank_without_process_group():
    sys.path.insert(0, ROOT)
    import bench
    t, v = bench.job_seconds_per_iter(2.5, steps=5)
    assert (t, v) == (2.5, 0.5)
