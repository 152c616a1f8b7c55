"""The bench's multi-rank logic on CPU: two gloo ranks agree on the slowest rank's time and the whole-job
throughput (weak scaling: every rank's units over that time); one rank needs no process group."""

import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        local_ms = [3.0, 5.0][rank]  # rank 1 is slower
        ms = bench.max_over_ranks(local_ms, ws, "cpu")
        out[rank] = (ms, bench.job_throughput(ws, 1e9, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for rank in (0, 1):
        ms, value = out[rank]
        assert ms == 5.0
        assert value == pytest.approx(2 * 1e9 / 5e-3 / 1e9)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.0, 1, "cpu") == 4.0
    assert bench.job_throughput(1, 134217728, 2.0) == pytest.approx(134217728 / 2e-3 / 1e9)
