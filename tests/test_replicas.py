"""Replicas (several GPUs, one process each, no data-path collective): the
job's rate uses the slowest rank's time.  Run as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    from paper_2402_04606_gb300.replicas import job_rate, max_over_ranks

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    slowest = max_over_ranks(1.0 + 0.5 * rank)  # rank r took 1 + r/2 seconds
    out[rank] = (slowest, job_rate(100.0, slowest, world))
    dist.destroy_process_group()


def test_slowest_rank_times_the_job():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (1.5, pytest.approx(200.0 / 1.5))


def test_single_process_is_identity():
    from paper_2402_04606_gb300.replicas import job_rate, max_over_ranks

    assert max_over_ranks(2.5) == 2.5
    assert job_rate(10.0, 2.0, 1) == 5.0
