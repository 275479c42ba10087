"""The multi-rank path of bench.py on CPU (gloo, world size 2): per-rank step times are
reduced to their maximum on every rank, and the whole-job rate counts every replica."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.max_over_ranks([100.0 * (rank + 1), 7.0 - rank], dist, "cpu")
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world_2():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == [200.0, 7.0] and out[1] == [200.0, 7.0]


def test_replica_rate_counts_every_rank():
    assert bench.replica_rate(1, 1, 0.5) == pytest.approx(2.0)
    assert bench.replica_rate(4, 1, 0.5) == pytest.approx(8.0)
    assert bench.replica_rate(2, 20, 300.0) == pytest.approx(40 / 300.0)
