"""The replica reduction of bench.py across two ranks (gloo, CPU).

Each rank runs its own structure; the job time is the slowest rank's and the throughput the
sum of all ranks' atoms over that time.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2407_06409_gb300.replicas import job_throughput
    secs = [2.0, 3.0][rank]
    atoms = [4096.0, 8192.0][rank]
    out[rank] = job_throughput(secs, atoms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_job_throughput():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        sec, thr = res[rank]
        assert sec == 3.0
        assert thr == pytest.approx((4096.0 + 8192.0) / 3.0)


def test_single_process_is_identity():
    from paper_2407_06409_gb300.replicas import job_throughput
    assert job_throughput(2.0, 100.0) == (2.0, 50.0)
