"""The multi-GPU path of bench.py is replicas only: the timed region's
duration is the maximum over ranks and the value is the whole-job rate.  Run
here as two gloo ranks on the CPU (one process per rank, 127.0.0.1)."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 * (rank + 1)                 # rank 1 is the slow one
    t = bench.max_over_ranks(local_ms, dist, device="cpu")
    rate = bench.whole_job_rate(1e6, 10, world, t)
    dist.barrier()
    out[rank] = (t, rate)
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_two_gloo_ranks():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]                        # every rank sees the same numbers
    t, rate = res[0]
    assert t == 200.0                              # the slowest rank's region
    assert rate == pytest.approx(1e6 * 10 * 2 / 0.2)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, device="cpu") == 12.5
    assert bench.whole_job_rate(3.0, 4, 1, 1000.0) == pytest.approx(12.0)
