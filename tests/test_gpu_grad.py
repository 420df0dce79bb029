"""GPU spatial gradient of the dipole sum (the oracle's reading R9: the x-gradient of
eq. dipole_sum and eq. farfield under the walk of Alg. 1) and its adjoint, vs
the oracle's double-precision Barnes-Hut on the same tree: forward norm-wise
error <= 1e-4 per channel and axis, adjoint <= 1e-3 (the tolerances of the
dipole sum and its adjoint)."""
import numpy as np
import pytest

import oracle
from paper_2405_16788_gb300 import synthetic as syn
from _helpers import bf16_round, gpu_tree, normwise, oracle_tree, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-4
TOL_ADJ = 1e-3


def _flat(g):
    """[Q, C, 3] -> [Q, 3C]: one column per channel and axis for normwise."""
    g = np.asarray(g)
    return g.reshape(g.shape[0], -1)


def _fwd(cloud, mu, queries, beta=2.0, leaf_size=8):
    gt = gpu_tree(cloud, leaf_size)
    gt.refit(to_dev(mu))
    q = to_dev(queries)
    d, gx = gt.forward_grad(q, beta)
    gt.sync_status()
    ot = oracle_tree(cloud, leaf_size)
    ot.update(mu)
    return gt, d.cpu().numpy(), gx.cpu().numpy(), ot


def test_forward_grad_sphere_2k():
    w = syn.workload("sphere-2k")
    gt, d, gx, ot = _fwd(w.cloud, w.mu, w.queries)
    ref = ot.forward_grad(w.queries, 2.0)
    assert gx.shape == ref.shape
    assert np.all(normwise(_flat(gx), _flat(ref)) <= TOL), normwise(_flat(gx), _flat(ref))
    # the value output is the dipole sum
    assert np.all(normwise(d, ot.forward(w.queries, 2.0)) <= TOL)
    assert np.all(normwise(d, gt.forward(to_dev(w.queries), 2.0).cpu().numpy()) <= 1e-5)


@pytest.mark.parametrize("C,beta", [(1, 2.0), (2, 1.0), (3, 2.0), (4, 4.0), (5, 2.0), (8, 2.0),
                                    (16, 0.5), (33, 2.0)])
def test_forward_grad_channels_and_betas(C, beta):
    w = syn.workload("scene-200k", scale=0.05)
    mu = syn.attributes(w.cloud.n, C, seed=C)
    q = w.queries[:6011]
    _, d, gx, ot = _fwd(w.cloud, mu, q, beta)
    assert gx.shape == (len(q), C, 3)
    ref = ot.forward_grad(q, beta)
    assert np.all(normwise(_flat(gx), _flat(ref)) <= TOL), normwise(_flat(gx), _flat(ref))
    assert np.all(normwise(d, ot.forward(q, beta)) <= TOL)


@pytest.mark.parametrize("leaf_size", [1, 16])
def test_forward_grad_leaf_sizes(leaf_size):
    w = syn.workload("scene-200k", scale=0.03)
    q = w.queries[:7000]
    _, _, gx, ot = _fwd(w.cloud, w.mu, q, leaf_size=leaf_size)
    ref = ot.forward_grad(q, 2.0)
    assert np.all(normwise(_flat(gx), _flat(ref)) <= TOL)


def test_forward_grad_no_far_node_is_brute_force():
    """beta -> infinity: the exact gradient, against the oracle's brute force."""
    w = syn.workload("sphere-2k", scale=0.5)
    c = w.cloud
    gt = gpu_tree(c)
    gt.refit(to_dev(w.mu))
    _, gx = gt.forward_grad(to_dev(w.queries), 1e30, value=False)
    bf = oracle.brute_forward_grad(c.points, c.normals, c.areas, c.eps, w.mu, w.queries)
    assert np.all(normwise(_flat(gx.cpu().numpy()), _flat(bf)) <= TOL)


def test_forward_grad_eps_zero_queries_on_points_and_near_points():
    """eps = 0 (singular kernel, no far-field cut) and queries exactly at points
    (the zero-distance term contributes nothing), plus queries within a few
    eps of points where the series branch is taken."""
    cl = syn.sphere_cloud(3000, seed=4, eps=None)
    mu = syn.attributes(cl.n, 2, seed=5, kind="unit01")
    q = np.concatenate([cl.points[:64], syn.uniform_box_queries(1000, seed=6)]).astype(np.float32)
    _, _, gx, ot = _fwd(cl, mu, q)
    assert np.all(np.isfinite(gx))
    ref = ot.forward_grad(q, 2.0)
    assert np.all(normwise(_flat(gx), _flat(ref)) <= TOL)
    w = syn.workload("scene-200k", scale=0.02)
    rng = np.random.default_rng(7)
    pick = rng.choice(w.cloud.n, 3000)
    eps = w.cloud.eps[pick][:, None]
    near = (w.cloud.points[pick] + rng.normal(size=(3000, 3)) * eps * rng.uniform(0.01, 3, (3000, 1)))
    near = near.astype(np.float32)
    _, _, gx, ot = _fwd(w.cloud, w.mu, near)
    ref = ot.forward_grad(near, 2.0)
    assert np.all(normwise(_flat(gx), _flat(ref)) <= TOL), normwise(_flat(gx), _flat(ref))


def test_forward_grad_bf16_attributes():
    """bf16 attributes: compared with the oracle on the same bf16-rounded values."""
    import torch
    w = syn.workload("scene-200k", scale=0.05)
    mu = syn.attributes(w.cloud.n, 4, seed=9)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(mu).to(torch.bfloat16))
    q = w.queries[:5000]
    _, gx = gt.forward_grad(to_dev(q), 2.0)
    ot = oracle_tree(w.cloud)
    ot.update(bf16_round(mu))
    ref = ot.forward_grad(q, 2.0)
    assert np.all(normwise(_flat(gx.cpu().numpy()), _flat(ref)) <= TOL)


def test_forward_grad_ragged_and_empty():
    import torch
    w = syn.workload("scene-200k", scale=0.02)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    ot = oracle_tree(w.cloud)
    ot.update(w.mu)
    for nq in (1, 31, 33, 1000):
        q = w.queries[:nq]
        _, gx = gt.forward_grad(to_dev(q), 2.0)
        assert np.all(normwise(_flat(gx.cpu().numpy()), _flat(ot.forward_grad(q, 2.0))) <= TOL)
    d, gx = gt.forward_grad(torch.zeros((0, 3), device="cuda"), 2.0)
    assert gx.shape == (0, 4, 3)
    gt.sync_status()


@pytest.mark.parametrize("C,with_g,with_G", [(4, True, True), (4, False, True), (3, True, True),
                                             (16, True, True), (1, False, True)])
def test_adjoint_grad(C, with_g, with_G):
    w = syn.workload("scene-200k", scale=0.05)
    mu = syn.attributes(w.cloud.n, C, seed=C + 20)
    q = w.queries[:20000]
    g = syn.upstream_grad(len(q), C, seed=3) if with_g else None
    G = np.random.default_rng(4).normal(size=(len(q), C, 3)).astype(np.float32) if with_G else None
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(mu))
    ga = gt.adjoint_grad(to_dev(q), 2.0, None if g is None else to_dev(g),
                         None if G is None else to_dev(G)).cpu().numpy()
    gt.sync_status()
    ot = oracle_tree(w.cloud)
    ot.update(mu)
    ref = ot.adjoint_grad(q, 2.0, None if g is None else g.astype(np.float64),
                          None if G is None else G.astype(np.float64))
    assert np.all(normwise(ga, ref) <= TOL_ADJ), normwise(ga, ref)


def test_adjoint_grad_value_part_is_the_adjoint():
    w = syn.workload("scene-200k", scale=0.05)
    q = to_dev(w.queries[:20000])
    g = to_dev(syn.upstream_grad(20000, 4, seed=5))
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    a = gt.adjoint(q, 2.0, g).cpu().numpy()
    b = gt.adjoint_grad(q, 2.0, g, None).cpu().numpy()
    assert np.all(normwise(b, a) <= 1e-5)


def test_adjoint_grad_identity_on_gpu():
    """<g, D> + <G, grad D> = <adjoint(g, G), mu>: both sides from GPU outputs."""
    w = syn.workload("scene-200k", scale=0.05)
    q = w.queries[:30000]
    g = syn.upstream_grad(len(q), 4, seed=6)
    G = np.random.default_rng(8).normal(size=(len(q), 4, 3)).astype(np.float32)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    d, gx = gt.forward_grad(to_dev(q), 2.0)
    dmu = gt.adjoint_grad(to_dev(q), 2.0, to_dev(g), to_dev(G)).cpu().numpy().astype(np.float64)
    d = d.cpu().numpy().astype(np.float64)
    gx = gx.cpu().numpy().astype(np.float64)
    lhs = np.sum(g * d) + np.sum(G * gx)
    rhs = np.sum(dmu * w.mu.astype(np.float64))
    scale = np.sum(np.abs(g * d)) + np.sum(np.abs(G * gx))
    assert abs(lhs - rhs) <= 1e-4 * scale, (lhs, rhs, scale)


def test_planned_grad_matches_unplanned():
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("scene-200k", scale=0.3)
    nq = 120000
    q = to_dev(w.queries[:nq])
    g = to_dev(syn.upstream_grad(nq, 4, seed=12))
    G = to_dev(np.random.default_rng(13).normal(size=(nq, 4, 3)).astype(np.float32))
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    d, gx = gt.forward_grad(q, 2.0)
    a = gt.adjoint_grad(q, 2.0, g, G).cpu().numpy()
    plan = dipole.QueryPlan(nq, q.device)
    dp, gxp = gt.forward_grad(q, 2.0, plan=plan)
    ap = gt.adjoint_grad(q, 2.0, g, G, plan=plan).cpu().numpy()
    assert np.array_equal(d.cpu().numpy(), dp.cpu().numpy())
    assert np.array_equal(gx.cpu().numpy(), gxp.cpu().numpy())
    assert np.all(normwise(ap, a) <= 1e-5)
    assert np.array_equal(np.sort(plan.perm.cpu().numpy()), np.arange(nq))
    gt.sync_status()


def test_autograd_of_sum_and_gradient():
    """dipole_sum_and_grad: backward equals adjoint_grad with the same upstream
    gradients; dipole_sum's query gradient equals sum_c dL/dD^c grad D^c from
    the oracle."""
    import torch
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("scene-200k", scale=0.03)
    q = w.queries[:8000]
    gt = gpu_tree(w.cloud)
    mu = to_dev(w.mu).requires_grad_(True)
    qd = to_dev(q)
    d, gx = dipole.dipole_sum_and_grad(mu, gt, qd, 2.0)
    wd = to_dev(syn.upstream_grad(len(q), 4, seed=14))
    wg = to_dev(np.random.default_rng(15).normal(size=(len(q), 4, 3)).astype(np.float32))
    ((d * wd).sum() + (gx * wg).sum()).backward()
    ref = gt.adjoint_grad(qd, 2.0, wd, wg).cpu().numpy()
    assert np.all(normwise(mu.grad.cpu().numpy(), ref) <= 1e-5)

    qv = to_dev(q).requires_grad_(True)
    mu2 = to_dev(w.mu).requires_grad_(True)
    y = dipole.dipole_sum(mu2, gt, qv, 2.0)
    (y * wd).sum().backward()
    ot = oracle_tree(w.cloud)
    ot.update(w.mu)
    gref = np.einsum("qc,qck->qk", wd.cpu().numpy().astype(np.float64), ot.forward_grad(q, 2.0))
    assert np.all(normwise(qv.grad.cpu().numpy(), gref) <= TOL), normwise(qv.grad.cpu().numpy(), gref)
    assert mu2.grad is not None


@pytest.mark.slow
def test_full_size_scene_1m_sampled_grad():
    """The benchmark's workload (1M points, 524,288 queries, C = 4): gradient
    of all queries on the GPU, 2048 sampled ones checked against the oracle;
    the adjoint with upstream gradients nonzero on the sample only."""
    w = syn.workload("scene-1m")
    Q = len(w.queries)
    idx = np.random.default_rng(2).choice(Q, 2048, replace=False)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    q = to_dev(w.queries)
    _, gx = gt.forward_grad(q, 2.0, value=False)
    gx = gx.cpu().numpy()
    G = np.zeros((Q, 4, 3), np.float32)
    G[idx] = np.random.default_rng(3).normal(size=(2048, 4, 3))
    ga = gt.adjoint_grad(q, 2.0, None, to_dev(G)).cpu().numpy()
    gt.sync_status()
    ot = oracle_tree(w.cloud)
    ot.update(w.mu)
    ref = ot.forward_grad(w.queries[idx], 2.0)
    assert np.all(normwise(_flat(gx[idx]), _flat(ref)) <= TOL), normwise(_flat(gx[idx]), _flat(ref))
    aref = ot.adjoint_grad(w.queries[idx], 2.0, None, G[idx].astype(np.float64))
    assert np.all(normwise(ga, aref) <= TOL_ADJ), normwise(ga, aref)
