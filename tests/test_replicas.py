"""The multi-GPU bench path runs independent replicas (one field per rank, no
data-path collective); its only cross-rank step is the timing reduction: the job
takes as long as its slowest rank, and the value counts every rank's bytes.  Checked
here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    steps = [[1.0, 2.0, 3.0], [2.0, 2.5, 4.5]][rank]  # totals 6 ms and 9 ms
    value, total = bench.whole_job(steps, world, 1_000_000, dist, torch.device("cpu"))
    out[rank] = (value, total)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        value, total = out[r]
        assert total == pytest.approx(9.0)
        # 2 ranks x 3 steps x 1 MB in 9 ms
        assert value == pytest.approx(2 * 3 * 1e6 / 9e-3 / 1e9)


def test_one_rank_needs_no_collective():
    import bench
    value, total = bench.whole_job([1.0, 1.0], 1, 4_000_000)
    assert total == pytest.approx(2.0) and value == pytest.approx(2 * 4e6 / 2e-3 / 1e9)
