"""The replica path of the benchmark (one process per GPU, each with its own frame and
table; no data-path collective): the timed region's aggregation over ranks, on CPU gloo
ranks (world size 2).  The slowest rank's time counts, and the whole-job rate is every
rank's units over that time."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs = [1.5, 4.0][rank]                       # rank 1 is the slow one
    dist.barrier()
    secs_max = bench.max_over_ranks(torch, dist, secs, "cpu")
    out[rank] = (secs_max, bench.whole_job_rate(1000, world, secs_max))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (4.0, 500.0)     # 2 ranks x 1000 units in the slowest 4 s


def test_single_process_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(torch, None, 2.5, "cpu") == 2.5
    assert bench.whole_job_rate(1000, 1, 2.5) == 400.0
