"""Multi-GPU is replicas only (every rank serves its own frames, no data-path exchange): the
host logic that turns per-rank windows into the job's throughput, run as two gloo ranks on the
CPU (the same calls bench.py makes over NCCL on GPUs)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, windows, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        el = bench.replica_window(dist, windows[rank])
        out[rank] = (el, bench.replica_throughput(100, world, el))
    finally:
        dist.destroy_process_group()


def test_replica_window_is_the_slowest_rank():
    world, port = 2, _free_port()
    windows = [0.25, 0.4]
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, windows, out), nprocs=world, start_method="spawn")
        got = dict(out)
    assert got[0] == got[1] == (0.4, 100 * 2 / 0.4)


def test_single_process_needs_no_group():
    assert bench.replica_window(None, 0.5) == 0.5
    assert bench.replica_throughput(1000, 1, 0.5) == 2000.0
