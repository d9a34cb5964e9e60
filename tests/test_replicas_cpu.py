"""Replicas across ranks (bench.py --gpus N): the whole-job time is the
slowest rank's and the work is the sum over ranks. Two gloo ranks on the CPU
exercise the reduction that the GPU run does over NCCL."""
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
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    try:
        # rank r: elapsed 10 + 5 r ms, 100 (r + 1) iterations
        out[rank] = bench.job_totals(10.0 + 5.0 * rank, 100 * (rank + 1), world, "cpu")
    finally:
        dist.destroy_process_group()


def test_job_totals_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        got = dict(out)
    assert got[0] == got[1] == (15.0, 300.0)


def test_job_totals_single_rank_is_identity():
    import bench
    assert bench.job_totals(12.5, 7, 1, "cpu") == (12.5, 7.0)
