"""Multi-GPU runs are independent replicas (the path has no sharded exchange on
one-GPU machines): the benchmark's whole-job figures are the slowest rank's time
and the sum of all ranks' entries.  Checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, entries = bench.aggregate_over_ranks(10.0 + 5.0 * rank, 1000 + rank)
    out[rank] = (ms, entries)
    dist.destroy_process_group()


def test_two_replicas_aggregate_with_gloo():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1] == (15.0, 2001)


def test_single_process_passthrough():
    import bench
    assert bench.aggregate_over_ranks(3.5, 42) == (3.5, 42)
