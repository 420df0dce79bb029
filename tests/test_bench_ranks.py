"""The multi-rank logic of bench.py on CPU (gloo, world size 2): every rank
gets its own batch of rays against the same point cloud, the job's time is
the slowest rank's, and the reported value counts the units of all ranks."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as td
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks(10.0 + 5.0 * rank, td)
        td.barrier()
    finally:
        td.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == 15.0 and out[1] == 15.0


def test_job_throughput_counts_every_rank():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5  # no process group: the value itself
    assert bench.job_throughput(4, 1000, 10, 20.0) == pytest.approx(4 * 1000 * 10 / 0.02)


def test_each_rank_gets_its_own_rays_on_the_same_cloud():
    import bench
    w0 = bench.rank_workload("scene-1m", 0)
    w1 = bench.rank_workload("scene-1m", 1)
    assert np.array_equal(w0.cloud.points, w1.cloud.points)
    assert w0.queries.shape == w1.queries.shape
    assert not np.array_equal(w0.queries, w1.queries)
