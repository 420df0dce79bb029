"""GPU adjoint (two-stage, Sec. 6.2) vs the oracle: norm-wise error <= 1e-3
against the oracle's double-precision Barnes-Hut adjoint on the same tree,
against brute force when nothing is far, the adjoint identity on the GPU,
and the autograd path against finite differences of a compositing loss
evaluated through the oracle in double precision."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_16788_gb300 import synthetic as syn
from _helpers import gpu_tree, normwise, oracle_tree, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-3


def _adj(cloud, mu, queries, g, beta=2.0, leaf_size=8):
    gt = gpu_tree(cloud, leaf_size)
    gt.refit(to_dev(mu))
    ga = gt.adjoint(to_dev(queries), beta, to_dev(g)).cpu().numpy()
    gt.sync_status()
    ot = oracle_tree(cloud, leaf_size)
    ot.update(mu)
    ref = ot.adjoint(queries, beta, g.astype(np.float64))
    return ga, ref, gt


def test_sphere_2k():
    w = syn.workload("sphere-2k")
    g = syn.upstream_grad(len(w.queries), 1, seed=1)
    ga, ref, _ = _adj(w.cloud, w.mu, w.queries, g)
    assert np.all(normwise(ga, ref) <= TOL), normwise(ga, ref)


@pytest.mark.parametrize("C,beta", [(4, 2.0), (1, 1.0), (3, 4.0), (16, 2.0), (33, 2.0), (40, 2.0)])
def test_scene(C, beta):
    w = syn.workload("scene-200k", scale=0.1)
    mu = syn.attributes(w.cloud.n, C, seed=C)
    q = w.queries[:40000]
    g = syn.upstream_grad(len(q), C, seed=2)
    ga, ref, _ = _adj(w.cloud, mu, q, g, beta)
    assert np.all(normwise(ga, ref) <= TOL), normwise(ga, ref)


@pytest.mark.parametrize("leaf_size", [1, 16])
def test_leaf_sizes(leaf_size):
    w = syn.workload("scene-200k", scale=0.03)
    q = w.queries[:9000]
    g = syn.upstream_grad(len(q), 4, seed=3)
    ga, ref, _ = _adj(w.cloud, w.mu, q, g, leaf_size=leaf_size)
    assert np.all(normwise(ga, ref) <= TOL)


def test_no_far_node_is_brute_force_adjoint():
    w = syn.workload("sphere-2k", scale=0.5)
    g = syn.upstream_grad(len(w.queries), 1, seed=4)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    ga = gt.adjoint(to_dev(w.queries), 1e30, to_dev(g)).cpu().numpy()
    c = w.cloud
    bf = oracle.brute_adjoint(c.points, c.normals, c.areas, c.eps, w.queries, g)
    assert np.all(normwise(ga, bf) <= TOL)


def test_accumulate_and_ragged():
    import torch
    w = syn.workload("scene-200k", scale=0.02)
    q = w.queries[:1237]
    g = syn.upstream_grad(len(q), 4, seed=5)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    a = gt.adjoint(to_dev(q), 2.0, to_dev(g))
    b = torch.full_like(a, 0.5)
    gt.adjoint(to_dev(q), 2.0, to_dev(g), grad_attrs=b, accumulate=True)
    assert torch.allclose(b, a + 0.5, rtol=0, atol=1e-6)
    z = gt.adjoint(torch.zeros((0, 3), device="cuda"), 2.0, torch.zeros((0, 4), device="cuda"))
    assert float(z.abs().max()) == 0.0
    gt.sync_status()


def test_adjoint_identity_on_gpu():
    """<g, K mu> = <K^T g, mu> with both sides computed by the GPU."""
    w = syn.workload("scene-200k", scale=0.1)
    q = w.queries[:50000]
    g = syn.upstream_grad(len(q), 4, seed=6)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    y = gt.forward(to_dev(q), 2.0).cpu().numpy().astype(np.float64)
    ga = gt.adjoint(to_dev(q), 2.0, to_dev(g)).cpu().numpy().astype(np.float64)
    lhs = np.sum(g * y)
    rhs = np.sum(ga * w.mu)
    scale = np.sum(np.abs(g * y))
    assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs, scale)


# ------------------------------------------------------- autograd + FD ------

S_SCALE = 50.0


def _render_loss_np(D, target, n_rays, n_samp):
    """Harness loss of a volume-rendering shape (Sec. 3.1, eqs. vacancy and
    quadrature): phi = 1/2 - D_geo, v = Phi(s phi), per-sample opacity from the
    change of v along the ray, colour = sum T alpha RGB, L1 to a target."""
    from scipy.special import ndtr
    D = D.reshape(n_rays, n_samp, -1)
    v = ndtr(S_SCALE * (0.5 - D[..., 0]))
    sd = np.abs(v[:, 1:] - v[:, :-1]) / np.maximum(v[:, 1:], 1e-6)
    alpha = np.concatenate([np.zeros((n_rays, 1)), 1 - np.exp(-sd)], axis=1)
    T = np.cumprod(np.concatenate([np.ones((n_rays, 1)), 1 - alpha[:, :-1]], axis=1), axis=1)
    col = np.sum((T * alpha)[..., None] * D[..., 1:4], axis=1)
    return np.sum(np.abs(col - target))


def _render_loss_torch(D, target, n_rays, n_samp):
    import torch
    D = D.reshape(n_rays, n_samp, -1)
    v = torch.special.ndtr(S_SCALE * (0.5 - D[..., 0]))
    sd = (v[:, 1:] - v[:, :-1]).abs() / v[:, 1:].clamp_min(1e-6)
    alpha = torch.cat([torch.zeros_like(v[:, :1]), 1 - torch.exp(-sd)], dim=1)
    T = torch.cumprod(torch.cat([torch.ones_like(v[:, :1]), 1 - alpha[:, :-1]], dim=1), dim=1)
    col = ((T * alpha)[..., None] * D[..., 1:4]).sum(dim=1)
    return (col - target).abs().sum()


def test_autograd_matches_finite_differences_of_oracle_loss():
    """The benchmark's differentiable workload shape at reduced size: gradient
    of a compositing loss w.r.t. all per-point attributes through the
    torch.autograd.Function, compared on 64 random points with central
    differences of the same loss evaluated through the oracle in double."""
    import torch
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("scene-1m", scale=0.03)
    o, d, t = w.meta["rays"]
    n_rays, n_samp = t.shape
    c = w.cloud
    mu_gt = w.mu
    mu = (mu_gt + np.random.default_rng(9).normal(scale=0.05, size=mu_gt.shape)).astype(np.float32)
    ot = oracle_tree(c)
    ot.update(mu_gt)
    target = ot.forward(w.queries, 2.0).reshape(n_rays, n_samp, -1)
    # target image rendered from the ground-truth attributes
    from scipy.special import ndtr
    tgt_col = None
    v = ndtr(S_SCALE * (0.5 - target[..., 0]))
    sd = np.abs(v[:, 1:] - v[:, :-1]) / np.maximum(v[:, 1:], 1e-6)
    alpha = np.concatenate([np.zeros((n_rays, 1)), 1 - np.exp(-sd)], axis=1)
    T = np.cumprod(np.concatenate([np.ones((n_rays, 1)), 1 - alpha[:, :-1]], axis=1), axis=1)
    tgt_col = np.sum((T * alpha)[..., None] * target[..., 1:4], axis=1)

    # GPU: autograd through DipoleSum
    gt = gpu_tree(c)
    attrs = to_dev(mu).requires_grad_(True)
    D = dipole.dipole_sum(attrs, gt, to_dev(w.queries), 2.0)
    L = _render_loss_torch(D, to_dev(tgt_col.astype(np.float32)), n_rays, n_samp)
    L.backward()
    grad = attrs.grad.cpu().numpy().astype(np.float64)

    # oracle: D(mu) and the columns K[:, m] for 64 points via one-hot channels
    ot.update(mu)
    D0 = ot.forward(w.queries, 2.0)
    rng = np.random.default_rng(10)
    pts = rng.choice(c.n, 64, replace=False)
    onehot = np.zeros((c.n, 64), np.float32)
    onehot[pts, np.arange(64)] = 1.0
    ot.update(onehot)
    K = ot.forward(w.queries, 2.0)  # [Q, 64]: column j = dD/dmu_{pts[j]} (any channel)
    h = 1e-4
    fd = np.zeros((64, 4))
    for j in range(64):
        for ch in range(4):
            Dp = D0.copy(); Dp[:, ch] += h * K[:, j]
            Dm = D0.copy(); Dm[:, ch] -= h * K[:, j]
            fd[j, ch] = (_render_loss_np(Dp, tgt_col, n_rays, n_samp) -
                         _render_loss_np(Dm, tgt_col, n_rays, n_samp)) / (2 * h)
    err = normwise(grad[pts], fd)
    assert np.all(err <= TOL), err


@pytest.mark.slow
def test_full_size_scene_1m_sampled_adjoint():
    """Benchmark workload and launch configuration (1M points, 524,288
    queries): upstream gradient nonzero on 4096 sampled queries only, so the
    oracle's adjoint over that sample is the full answer."""
    w = syn.workload("scene-1m")
    Q = len(w.queries)
    idx = np.random.default_rng(1).choice(Q, 4096, replace=False)
    g = np.zeros((Q, 4), np.float32)
    g[idx] = syn.upstream_grad(4096, 4, seed=11)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    ga = gt.adjoint(to_dev(w.queries), 2.0, to_dev(g)).cpu().numpy()
    gt.sync_status()
    ot = oracle_tree(w.cloud)
    ot.update(w.mu)
    ref = ot.adjoint(w.queries[idx], 2.0, g[idx].astype(np.float64))
    assert np.all(normwise(ga, ref) <= TOL), normwise(ga, ref)


def test_planned_forward_and_adjoint_match_unplanned():
    """The query plan (Morton order + packet costs written by the forward)
    changes only the order of work: results equal the plain calls', also when
    the plan came from a different query batch of the same size."""
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("scene-200k", scale=0.3)  # enough packets for longest-first scheduling
    q = to_dev(w.queries[:120000])
    g = to_dev(syn.upstream_grad(120000, 4, seed=12))
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    y = gt.forward(q, 2.0).cpu().numpy()
    a = gt.adjoint(q, 2.0, g).cpu().numpy()
    plan = dipole.QueryPlan(120000, q.device)
    yp = gt.forward(q, 2.0, plan=plan).cpu().numpy()
    ap = gt.adjoint(q, 2.0, g, plan=plan).cpu().numpy()
    assert np.array_equal(y, yp)
    assert np.all(normwise(ap, a) <= 1e-5)
    perm = plan.perm.cpu().numpy()
    assert np.array_equal(np.sort(perm), np.arange(120000))
    # a plan made on other queries of the same size
    q2 = to_dev(w.queries[150000:270000])
    gt.forward(q2, 2.0, plan=plan)
    ap2 = gt.adjoint(q, 2.0, g, plan=plan).cpu().numpy()
    assert np.all(normwise(ap2, a) <= 1e-5)
    gt.sync_status()


def test_planned_adjoint_with_any_plan_record_is_correct():
    """The adjoint cuts each packet's walk at the plan's recorded nodes; any
    record (here random words: non-increasing cuts, out-of-range nodes, keys
    of any size) only changes how the work is divided, never the result."""
    import torch
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("scene-200k", scale=0.3)
    nq = 120000
    q = to_dev(w.queries[:nq])
    g = to_dev(syn.upstream_grad(nq, 4, seed=13))
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    ref = gt.adjoint(q, 2.0, g).cpu().numpy()
    plan = dipole.QueryPlan(nq, q.device)
    gt.forward(q, 2.0, plan=plan)  # a valid permutation
    gen = torch.Generator(device="cuda").manual_seed(3)
    nn = gt.info["n_nodes"]
    for lo, hi in [(0, 2 ** 31 - 1), (0, nn), (0, 4000)]:
        plan.cost.copy_(torch.randint(lo, hi, plan.cost.shape, generator=gen, device="cuda",
                                      dtype=torch.int64).to(torch.int32))
        got = gt.adjoint(q, 2.0, g, plan=plan).cpu().numpy()
        assert np.all(normwise(got, ref) <= 1e-5), normwise(got, ref)
    gt.sync_status()
