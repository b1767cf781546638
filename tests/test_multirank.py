"""The benchmark's multi-rank path on CPU with gloo, world size 2: each rank
runs its own replicas; the job value is all ranks' solves over the slowest
rank's time, and the reference arm prints from rank 0 only."""
import io
import contextlib
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, solves = bench.combine_ranks(10.0 * (rank + 1), 7, dist, torch.device("cpu"))
    out[rank] = (ms, solves)
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_gloo_world2():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == (20.0, 14)   # max time, summed solves


def test_combine_ranks_single_process():
    import bench
    assert bench.combine_ranks(5.0, 3) == (5.0, 3)


def test_reference_arm_prints_on_rank0_only():
    import bench

    class A:
        steps, warmup, tol, gpus = 1, 0, 1e-8, 2
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(A, rank=1, world=2) == 0
    assert buf.getvalue() == ""
