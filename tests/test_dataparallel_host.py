"""Host logic of the data-parallel adjoint (paper_2405_16788_gb300/dataparallel.py)
on CPU: two gloo ranks hold disjoint halves of a query batch; each runs stage 1
on its half, the stage-1 sums are all-reduced, stage 2 runs on the sum.  A
stand-in tree whose stage 1 is the oracle's FP64 adjoint on the rank's queries
(stage 2 the identity: the oracle's adjoint already includes it, and both
stages are linear in the upstream gradient) checks that every rank ends with
the adjoint over all queries, to FP64 rounding."""
import os
import socket
import sys

import numpy as np
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _OracleTree:
    def __init__(self, ot):
        self.ot = ot

    def adjoint_stage1(self, queries, beta, grad_out, plan=None):
        g = self.ot.adjoint(queries.numpy(), beta, grad_out.numpy().astype(np.float64))
        return torch.from_numpy(np.ascontiguousarray(g).reshape(-1))

    def adjoint_stage2(self, acc, grad_attrs=None):
        return acc.reshape(self.ot.n, -1)


def _case():
    from paper_2405_16788_gb300 import synthetic as syn
    w = syn.workload("sphere-2k")
    g = syn.upstream_grad(len(w.queries), 1, seed=9)
    return w, g


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as td
    import oracle
    from paper_2405_16788_gb300 import dataparallel
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, g = _case()
        c = w.cloud
        ot = oracle.Tree(c.points, c.normals, c.areas, c.eps)
        ot.update(w.mu)
        half = slice(rank * len(w.queries) // world, (rank + 1) * len(w.queries) // world)
        res = dataparallel.adjoint_data_parallel(_OracleTree(ot), torch.from_numpy(w.queries[half]),
                                                 2.0, torch.from_numpy(g[half]))
        out[rank] = res.numpy().copy()
        td.barrier()
    finally:
        td.destroy_process_group()


def test_data_parallel_adjoint_gloo_world2_equals_single_rank():
    import oracle
    oracle.build()
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    w, g = _case()
    c = w.cloud
    ot = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    ot.update(w.mu)
    ref = ot.adjoint(w.queries, 2.0, g.astype(np.float64))
    for r in (0, 1):
        assert np.allclose(out[r], ref, rtol=1e-12, atol=1e-15 * np.abs(ref).max())
    # each rank's half alone is not the whole
    assert not np.allclose(ot.adjoint(w.queries[:len(w.queries) // 2], 2.0,
                                      g[:len(w.queries) // 2].astype(np.float64)), ref)


def test_all_reduce_sum_without_a_process_group_is_the_identity():
    from paper_2405_16788_gb300 import dataparallel
    a = torch.arange(5.0)
    assert dataparallel.all_reduce_sum(a) is a
    assert torch.equal(a, torch.arange(5.0))
