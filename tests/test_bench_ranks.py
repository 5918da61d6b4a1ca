"""The N-rank path of bench.py on CPU: two gloo ranks (replicas of the local
stage, no data-path collective) agree on the slowest rank's time, and the
whole-job rate counts the units of every rank over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank                      # rank 1 is the slow one
    worst = bench.max_over_ranks(ms, world, torch.device("cpu"))
    dist.barrier()
    out[rank] = (worst, bench.job_rate(world, 32, 3, worst))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    worst, rate = res[0]
    assert worst == 150.0
    assert rate == pytest.approx(2 * 32 * 3 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5, 1, None) == 12.5
    assert bench.job_rate(1, 32, 3, 1000.0) == pytest.approx(96.0)
