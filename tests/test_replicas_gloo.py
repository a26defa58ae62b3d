"""Multi-GPU path of the bench (replicas only: no data-path collective) on CPU ranks:
two gloo processes, max-over-ranks time and whole-job throughput."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(times[rank], dist, "cpu")
    out[rank] = (ms, bench.replica_throughput(3.0e6, world, ms))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_sum_the_work():
    import torch.multiprocessing as mp
    port = _free_port()
    times = [120.0, 250.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, times, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    for r in (0, 1):
        ms, value = res[r]
        assert ms == 250.0
        assert value == pytest.approx(2 * 3.0e6 / 0.25 / 1e9)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.replica_throughput(1e9, 1, 1000.0) == pytest.approx(1.0)
