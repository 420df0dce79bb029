"""GPU adjoint with respect to the normals and radii (the oracle's reading R10) vs the
oracle's double-precision Barnes-Hut on the same tree: norm-wise error <= 1e-3
per column (the adjoint tolerance), for upstream gradients of D, of grad D,
or both; the linearity identity on the GPU; the autograd path."""
import numpy as np
import pytest

import oracle
from paper_2405_16788_gb300 import synthetic as syn
from _helpers import bf16_round, gpu_tree, normwise, oracle_tree, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-3


def _upstream(nq, C, seed, with_g=True, with_G=True):
    rng = np.random.default_rng(seed)
    g = rng.normal(size=(nq, C)).astype(np.float32) if with_g else None
    G = rng.normal(size=(nq, C, 3)).astype(np.float32) if with_G else None
    return g, G


def _gpu_geom(gt, q, g, G, **kw):
    gm, gn, ge = gt.adjoint_geom(to_dev(q), 2.0 if "beta" not in kw else kw.pop("beta"),
                                 None if g is None else to_dev(g), None if G is None else to_dev(G),
                                 **kw)
    gt.sync_status()
    f = lambda t: None if t is None else t.cpu().numpy()
    return f(gm), f(gn), f(ge)


def _err(y, ref):
    """normwise, except that a column whose oracle values all lie below the
    float range (|ref| < 1e-30: e.g. exp(-t^2) factors of far-away points,
    nonzero only in double) is compared with an absolute bound of 1e-30."""
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    if y.ndim == 1:
        y, ref = y[:, None], ref[:, None]
    den = np.maximum(np.max(np.abs(ref), axis=0), 1e-30)
    return np.max(np.abs(y - ref), axis=0) / den


def _check(got, ref):
    gm, gn, ge = got
    rm, rn, re = ref
    if gm is not None:
        assert np.all(_err(gm, rm) <= TOL), _err(gm, rm)
    if gn is not None:
        assert np.all(_err(gn, rn) <= TOL), _err(gn, rn)
    if ge is not None:
        assert np.all(_err(ge, re) <= TOL), _err(ge, re)


@pytest.mark.parametrize("C,with_g,with_G,beta", [(4, True, True, 2.0), (4, True, False, 2.0),
                                                  (4, False, True, 1.0), (1, True, True, 2.0),
                                                  (3, True, True, 4.0), (16, True, True, 2.0)])
def test_adjoint_geom_matches_oracle(C, with_g, with_G, beta):
    w = syn.workload("scene-200k", scale=0.05)
    mu = syn.attributes(w.cloud.n, C, seed=C + 30)
    q = w.queries[:20000]
    g, G = _upstream(len(q), C, seed=C, with_g=with_g, with_G=with_G)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(mu))
    got = _gpu_geom(gt, q, g, G, beta=beta)
    ot = oracle_tree(w.cloud)
    ot.update(mu)
    ref = ot.adjoint_geom(q, beta, None if g is None else g.astype(np.float64),
                          None if G is None else G.astype(np.float64))
    _check(got, ref)


def test_adjoint_geom_no_far_node_is_brute_force():
    w = syn.workload("sphere-2k", scale=0.5)
    c = w.cloud
    g, G = _upstream(len(w.queries), 1, seed=3)
    gt = gpu_tree(c)
    gt.refit(to_dev(w.mu))
    got = _gpu_geom(gt, w.queries, g, G, beta=1e30)
    ref = oracle.brute_adjoint_geom(c.points, c.normals, c.areas, c.eps, w.mu, w.queries,
                                    g.astype(np.float64), G.astype(np.float64))
    _check(got, ref)


def test_adjoint_geom_eps_zero_and_queries_on_points():
    cl = syn.sphere_cloud(3000, seed=4, eps=None)
    mu = syn.attributes(cl.n, 2, seed=5, kind="unit01")
    q = np.concatenate([cl.points[:64], syn.uniform_box_queries(2000, seed=6)]).astype(np.float32)
    g, G = _upstream(len(q), 2, seed=7)
    gt = gpu_tree(cl)
    gt.refit(to_dev(mu))
    gm, gn, ge = _gpu_geom(gt, q, g, G)
    assert np.all(ge == 0.0)
    ot = oracle_tree(cl)
    ot.update(mu)
    rm, rn, _ = ot.adjoint_geom(q, 2.0, g.astype(np.float64), G.astype(np.float64))
    _check((gm, gn, None), (rm, rn, None))


def test_adjoint_geom_bf16_attributes():
    import torch
    w = syn.workload("scene-200k", scale=0.05)
    mu = syn.attributes(w.cloud.n, 4, seed=9)
    q = w.queries[:10000]
    g, G = _upstream(len(q), 4, seed=10)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(mu).to(torch.bfloat16))
    got = _gpu_geom(gt, q, g, G)
    ot = oracle_tree(w.cloud)
    ot.update(bf16_round(mu))
    _check(got, ot.adjoint_geom(q, 2.0, g.astype(np.float64), G.astype(np.float64)))


def test_adjoint_geom_attr_part_and_linearity_on_gpu():
    """The attribute output equals adjoint_grad's; sum_m n_m . dL/dn_m equals
    <g, D> + <G, grad D> (D is linear in the normals), all from GPU outputs."""
    w = syn.workload("scene-200k", scale=0.05)
    q = w.queries[:30000]
    g, G = _upstream(len(q), 4, seed=11)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    gm, gn, _ = _gpu_geom(gt, q, g, G)
    ga = gt.adjoint_grad(to_dev(q), 2.0, to_dev(g), to_dev(G)).cpu().numpy()
    assert np.all(normwise(gm, ga) <= 1e-5)
    d, gx = gt.forward_grad(to_dev(q), 2.0)
    lhs = np.sum(g.astype(np.float64) * d.cpu().numpy()) + np.sum(G.astype(np.float64) * gx.cpu().numpy())
    rhs = np.sum(w.cloud.normals.astype(np.float64) * gn)
    assert abs(lhs - rhs) <= 1e-4 * np.sum(np.abs(w.cloud.normals * gn)), (lhs, rhs)


def test_adjoint_geom_ragged_empty_and_accumulate():
    import torch
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("scene-200k", scale=0.02)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    ot = oracle_tree(w.cloud)
    ot.update(w.mu)
    for nq in (1, 33, 1000):
        q = w.queries[:nq]
        g, G = _upstream(nq, 4, seed=nq)
        _check(_gpu_geom(gt, q, g, G), ot.adjoint_geom(q, 2.0, g.astype(np.float64),
                                                        G.astype(np.float64)))
    # q = 0 writes zeros; accumulate = 1 adds
    n = w.cloud.n
    gn = torch.full((n, 3), 2.0, device="cuda")
    ge = torch.full((n,), 3.0, device="cuda")
    q0 = torch.zeros((0, 3), device="cuda")
    dipole.dipole_adjoint_geom(gt.handle, q0, 2.0, None, None, None, gn, ge, accumulate=True)
    assert torch.all(gn == 2.0) and torch.all(ge == 3.0)
    dipole.dipole_adjoint_geom(gt.handle, q0, 2.0, None, None, None, gn, ge, accumulate=False)
    assert torch.all(gn == 0.0) and torch.all(ge == 0.0)
    q = w.queries[:500]
    g, G = _upstream(500, 4, seed=1)
    base = torch.ones((n, 3), device="cuda")
    dipole.dipole_adjoint_geom(gt.handle, to_dev(q), 2.0, to_dev(g), to_dev(G), None, base, None,
                               accumulate=True)
    _, rn, _ = ot.adjoint_geom(q, 2.0, g.astype(np.float64), G.astype(np.float64))
    assert np.all(normwise(base.cpu().numpy() - 1.0, rn) <= TOL)
    gt.sync_status()


def test_planned_geom_matches_unplanned():
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("scene-200k", scale=0.3)
    nq = 120000
    q = to_dev(w.queries[:nq])
    g, G = _upstream(nq, 4, seed=12)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    a = gt.adjoint_geom(q, 2.0, to_dev(g), to_dev(G))
    plan = dipole.QueryPlan(nq, q.device)
    gt.forward_grad(q, 2.0, plan=plan)
    b = gt.adjoint_geom(q, 2.0, to_dev(g), to_dev(G), plan=plan)
    for u, v in zip(a, b):
        u = u.cpu().numpy()
        v = v.cpu().numpy()
        if u.ndim == 1:
            u, v = u[:, None], v[:, None]
        assert np.all(normwise(v, u) <= 1e-5)
    gt.sync_status()


def test_dipole_field_autograd():
    """dipole_field: gradients of normals, radii and attributes equal the
    adjoint's; the global-eps derivative of a loss through the oracle's FP64
    Barnes-Hut (central differences) equals the sum of the radius gradients."""
    import torch
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("scene-200k", scale=0.02)
    c = w.cloud
    n = c.n
    eps0 = 0.01
    radii = np.full(n, eps0, np.float32)
    P, A = to_dev(c.points), to_dev(c.areas)
    N = to_dev(c.normals).requires_grad_(True)
    E = to_dev(radii).requires_grad_(True)
    M = to_dev(w.mu).requires_grad_(True)
    q = w.queries[:6000]
    Q = to_dev(q)
    g, G = _upstream(len(q), 4, seed=13)
    d, gx = dipole.dipole_field(P, N, A, E, M, Q, 2.0, with_grad=True)
    ((d * to_dev(g)).sum() + (gx * to_dev(G)).sum()).backward()
    gt = dipole.DipoleTree(P, to_dev(c.normals), A, to_dev(radii))
    gt.refit(to_dev(w.mu))
    rm, rn, re = gt.adjoint_geom(Q, 2.0, to_dev(g), to_dev(G))
    assert np.all(normwise(M.grad.cpu().numpy(), rm.cpu().numpy()) <= 1e-5)
    assert np.all(normwise(N.grad.cpu().numpy(), rn.cpu().numpy()) <= 1e-5)
    assert np.all(normwise(E.grad.cpu().numpy()[:, None], re.cpu().numpy()[:, None]) <= 1e-5)

    def loss(e):
        ot = oracle.Tree(c.points, c.normals, c.areas, np.full(n, e, np.float32))
        ot.update(w.mu)
        return (np.sum(g.astype(np.float64) * ot.forward(q, 2.0)) +
                np.sum(G.astype(np.float64) * ot.forward_grad(q, 2.0)))

    h = 1e-6
    ep, em = np.float32(eps0 + h), np.float32(eps0 - h)
    fd = (loss(ep) - loss(em)) / (float(ep) - float(em))
    total = float(E.grad.double().sum())
    assert abs(total - fd) <= 1e-3 * abs(fd), (total, fd)


@pytest.mark.slow
def test_full_size_scene_1m_sampled_geom():
    """The benchmark's workload (1M points, 524,288 queries, C = 4): upstream
    gradients nonzero on 2048 sampled queries, so the oracle's adjoint over the
    sample is the full answer."""
    w = syn.workload("scene-1m")
    Q = len(w.queries)
    idx = np.random.default_rng(4).choice(Q, 2048, replace=False)
    g = np.zeros((Q, 4), np.float32)
    G = np.zeros((Q, 4, 3), np.float32)
    gs, Gs = _upstream(2048, 4, seed=14)
    g[idx], G[idx] = gs, Gs
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    got = _gpu_geom(gt, w.queries, g, G)
    ot = oracle_tree(w.cloud)
    ot.update(w.mu)
    _check(got, ot.adjoint_geom(w.queries[idx], 2.0, gs.astype(np.float64), Gs.astype(np.float64)))
