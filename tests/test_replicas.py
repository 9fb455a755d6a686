"""Replica aggregation across ranks (world_size 2, gloo, CPU): the whole-job
throughput is the sum of the ranks' work over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2606_10477_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, seconds = (8.0, 2.0) if rank == 0 else (8.0, 4.0)
    value, tmax, total = replicas.aggregate(units, seconds, dist)
    out[rank] = (value, tmax, total, replicas.rank_seed(1, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of this (multi-threaded) process
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        value, tmax, total, seed = res[rank]
        assert tmax == 4.0 and total == 16.0 and value == 4.0
    assert res[0][3] != res[1][3]


def test_single_process_is_local():
    assert replicas.aggregate(10.0, 2.0, None) == (5.0, 2.0, 10.0)
