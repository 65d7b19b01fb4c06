"""The multi-GPU path of the benchmark is replicas (one evaluation stream per
rank, no collective on the data path); the only cross-rank step is the
timing reduction.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) * 100 ms for its 10 evaluations
        rate, ms = bench.job_rate(10, (rank + 1) * 100.0, world)
        out[rank] = (rate, ms)
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    for r in range(world):
        rate, ms = res[r]
        assert ms == 200.0  # max over ranks
        assert rate == pytest.approx(world * 10 / 0.2)  # all ranks' units / slowest time


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.job_rate(4, 500.0, 1) == (8.0, 500.0)
