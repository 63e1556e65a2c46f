"""The multi-rank path of bench.py on CPU (gloo, world size 2).

Each rank runs its own replica of the workload (the ranks exchange no data);
the job's time is the slowest rank's and its rate is all ranks' updates over
that time.  Here the two ranks report different times and the same number of
updates, and both must get the slowest time and the whole-job rate."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms, value = bench.job_rate(10.0 * (rank + 1), world, 1e9)
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank():
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 20.0
        assert value == pytest.approx(2e9 / 0.020)


def test_job_rate_single_rank():
    import bench
    ms, value = bench.job_rate(8.0, 1, 4e9)
    assert ms == 8.0 and value == pytest.approx(5e11)
