"""The data-parallel adjoint (paper_2405_16788_gb300/dataparallel.py) with two
gloo ranks sharing one GPU: each rank builds the same tree, runs stage 1 of the
adjoint on its half of the queries into its own accumulator, the accumulators
are all-reduced on host copies (no NCCL, no device collective: no kernel waits
on another rank), and stage 2 runs on the sum.  Every rank's result equals the
single-rank adjoint over all queries to 1e-5 (the order of float sums)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs():
    from paper_2405_16788_gb300 import synthetic as syn
    w = syn.workload("scene-200k", scale=0.1)
    g = syn.upstream_grad(len(w.queries), w.mu.shape[1], seed=17)
    return w, g


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as td
    from paper_2405_16788_gb300 import dataparallel, dipole
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, g = _inputs()
        c = w.cloud
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        tree = dipole.DipoleTree(t(c.points), t(c.normals), t(c.areas), t(c.eps))
        tree.refit(t(w.mu))
        Q = len(w.queries)
        mine = slice(rank * Q // world, (rank + 1) * Q // world)
        res = dataparallel.adjoint_data_parallel(tree, t(w.queries[mine]), 2.0, t(g[mine]))
        tree.sync_status()
        out[rank] = res.cpu().numpy()
        td.barrier()
    finally:
        td.destroy_process_group()


def test_data_parallel_adjoint_two_ranks_one_gpu():
    import torch
    from paper_2405_16788_gb300 import dipole
    from _helpers import normwise
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    w, g = _inputs()
    c = w.cloud
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    tree = dipole.DipoleTree(t(c.points), t(c.normals), t(c.areas), t(c.eps))
    tree.refit(t(w.mu))
    ref = tree.adjoint(t(w.queries), 2.0, t(g)).cpu().numpy()
    tree.sync_status()
    for r in (0, 1):
        assert np.all(normwise(out[r], ref) <= 1e-5), normwise(out[r], ref)
