"""The replicas path of bench.py on CPU: two gloo ranks, each with its own
time; the job's time is the slowest rank's and its rate counts the units of
both ranks (weak scaling).  The data path itself has no collective."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_max = bench.max_over_ranks(times[rank])
    dist.barrier()
    out[rank] = (ms_max, bench.job_rate(world, 10, ms_max))
    dist.destroy_process_group()


def test_two_ranks_max_time_and_job_rate():
    world = 2
    times = [120.0, 150.0]
    # The free port is released before the ranks bind it, so another process
    # can take it in between: the rendezvous is retried on a fresh port.
    for attempt in range(3):
        port = _free_port()
        try:
            with mp.Manager() as man:
                out = man.dict()
                mp.spawn(_rank, args=(world, port, times, out), nprocs=world, join=True)
                res = dict(out)
            break
        except Exception:
            if attempt == 2:
                raise
    for r in range(world):
        ms_max, rate = res[r]
        assert ms_max == 150.0
        assert rate == pytest.approx(2 * 10 / 0.150)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(1, 50, 250.0) == pytest.approx(200.0)
