"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas) combine their
timings by the maximum over ranks, and the job's value counts the units of
every rank over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = [10.0 + 5.0 * rank, 0.5 - 0.25 * rank]   # rank 1 is slower on device, faster e2e
    out[rank] = bench.max_over_ranks(dist, mine, "cpu")
    dist.destroy_process_group()


def test_two_ranks_take_the_maximum():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == [15.0, 0.5]


def test_value_and_single_rank():
    import bench
    assert bench.max_over_ranks(None, [3.0, 4.0], "cpu") == [3.0, 4.0]
    # 2 ranks x 1 evaluation x 100 steps over the slowest rank's 250 ms
    assert bench.job_value(2, 1, 100, 250.0) == pytest.approx(800.0)
