"""The adjoint's two stages as separate calls (Sec. 6.2, App. C), the query-
position chain rule summed in the library, and the per-packet warp counts.

* dipole_adjoint_stage1 on two halves of a query batch into one accumulator,
  then dipole_adjoint_stage2, equals dipole_adjoint over the whole batch (the
  stages are linear; only the order of float sums differs: 1e-5), with and
  without a query plan; and equals the oracle's FP64 adjoint (1e-3).
* dipole_adjoint_queries equals sum_c g^c grad D^c of the oracle's FP64
  Barnes-Hut spatial gradient (the gradient gate, 1e-3 per axis) and of
  dipole_forward_grad on the same GPU (1e-5).
* dipole_query_packet_counts: the warp steps of each packet equal the steps
  that the forward's query plan recorded for it (the union of its lanes'
  walks does not depend on how the walk is cut into ranges); per-query
  counts equal dipole_query_counts; far steps <= steps; every packet walks at
  least as many steps as its longest lane."""
import numpy as np
import pytest
import torch

from paper_2405_16788_gb300 import synthetic as syn
from _helpers import gpu_tree, normwise, oracle_tree, to_dev

pytestmark = pytest.mark.gpu


def _setup(C=4, scale=0.1, nq=None):
    w = syn.workload("scene-200k", scale=scale)
    mu = syn.attributes(w.cloud.n, C, seed=31)
    q = w.queries if nq is None else w.queries[:nq]
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(mu))
    return w, mu, q, gt


@pytest.mark.parametrize("nq", [3001, None])  # below and above the ranged-item threshold
def test_stage1_halves_then_stage2_equal_adjoint(nq):
    from paper_2405_16788_gb300 import dipole
    w, mu, q, gt = _setup(nq=nq)
    Q, C = len(q), mu.shape[1]
    g = syn.upstream_grad(Q, C, seed=5)
    X, G = to_dev(q), to_dev(g)
    full = gt.adjoint(X, 2.0, G).cpu().numpy()
    h = Q // 2
    acc = gt.adjoint_stage1(X[:h], 2.0, G[:h])
    assert acc.numel() == gt.adjoint_acc_size()
    gt.adjoint_stage1(X[h:], 2.0, G[h:], acc=acc, accumulate=True)
    split = gt.adjoint_stage2(acc).cpu().numpy()
    assert np.all(normwise(split, full) <= 1e-5), normwise(split, full)
    # with the plan of a forward on the same (whole) batch
    plan = dipole.QueryPlan(Q, X.device)
    gt.forward(X, 2.0, plan=plan)
    acc2 = gt.adjoint_stage1(X, 2.0, G, plan=plan)
    planned = gt.adjoint_stage2(acc2).cpu().numpy()
    assert np.all(normwise(planned, full) <= 1e-5)
    # stage 2 with accumulate adds
    base = torch.ones((gt.n, C), device=X.device)
    gt.adjoint_stage2(acc2, grad_attrs=base, accumulate=True)
    assert np.all(normwise(base.cpu().numpy() - 1.0, full) <= 1e-5)
    gt.sync_status()
    ot = oracle_tree(w.cloud)
    ot.update(mu)
    ref = ot.adjoint(q, 2.0, g.astype(np.float64))
    assert np.all(normwise(split, ref) <= 1e-3), normwise(split, ref)


@pytest.mark.parametrize("C,nq", [(1, 5000), (4, None), (6, 7001)])
def test_adjoint_queries_is_the_chain_rule(C, nq):
    w, mu, q, gt = _setup(C=C, nq=nq)
    Q = len(q)
    g = syn.upstream_grad(Q, C, seed=6)
    X = to_dev(q)
    gq = gt.adjoint_queries(X, 2.0, to_dev(g)).cpu().numpy()
    _, gx = gt.forward_grad(X, 2.0, value=False)
    dev_ref = np.einsum("qc,qck->qk", g.astype(np.float64), gx.cpu().numpy().astype(np.float64))
    assert np.all(normwise(gq, dev_ref) <= 1e-5), normwise(gq, dev_ref)
    gt.sync_status()
    idx = np.random.default_rng(C).choice(Q, min(Q, 3000), replace=False)
    ot = oracle_tree(w.cloud)
    ot.update(mu)
    ref = np.einsum("qc,qck->qk", g[idx].astype(np.float64), ot.forward_grad(q[idx], 2.0))
    assert np.all(normwise(gq[idx], ref) <= 1e-3), normwise(gq[idx], ref)


def test_packet_counts_match_plan_and_query_counts():
    from paper_2405_16788_gb300 import dipole
    w, mu, q, gt = _setup()
    Q = len(q)
    assert Q >= 65536  # the forward runs ranged items: the plan's steps add two items
    X = to_dev(q)
    npk = (Q + 31) // 32
    pc = torch.empty((npk, 4), dtype=torch.int32, device=X.device)
    cnt = torch.empty((Q, 3), dtype=torch.int32, device=X.device)
    dipole.dipole_query_packet_counts(gt.handle, X, 2.0, pc, counts=cnt)
    ref_cnt = gt.query_counts(X, 2.0)
    plan = dipole.QueryPlan(Q, X.device)
    gt.forward(X, 2.0, plan=plan)
    gt.sync_status()
    pc, cnt, ref_cnt = pc.cpu().numpy(), cnt.cpu().numpy(), ref_cnt.cpu().numpy()
    assert np.array_equal(cnt, ref_cnt)
    steps = plan.cost.cpu().numpy().reshape(npk, -1)[:, 0]
    assert np.array_equal(pc[:, 0], steps)
    assert np.all(pc[:, 1] <= pc[:, 0])
    assert pc[:, 3].sum() == Q and np.all(pc[:-1, 3] == 32)
    # a packet's lanes are its 32 consecutive queries in the sort order
    perm = plan.perm.cpu().numpy()[:Q]
    longest = np.zeros(npk, np.int64)
    np.maximum.at(longest, np.arange(Q) // 32, cnt[perm, 0])
    assert np.all(pc[:, 0] >= longest)
