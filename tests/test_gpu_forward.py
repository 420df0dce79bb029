"""GPU primal queries vs the oracle's double-precision Barnes-Hut on the same
tree: norm-wise error <= 1e-4 per channel, traversal decisions (per-query
counts of tested nodes, far nodes and leaf points) bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2405_16788_gb300 import synthetic as syn
from _helpers import bf16_round, excess_over_allowance, gpu_tree, normwise, oracle_tree, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _run(cloud, mu, queries, beta=2.0, leaf_size=8, max_depth=10, counts=True):
    import torch
    gt = gpu_tree(cloud, leaf_size, max_depth)
    gt.refit(to_dev(mu))
    q = to_dev(queries)
    y = gt.forward(q, beta).cpu().numpy()
    c = gt.query_counts(q, beta).cpu().numpy() if counts else None
    gt.sync_status()
    ot = oracle_tree(cloud, leaf_size, max_depth)
    ot.update(mu)
    ref, rc = ot.forward(queries, beta, counters=True)
    return y, ref, c, rc


def test_sphere_2k():
    w = syn.workload("sphere-2k")
    y, ref, c, rc = _run(w.cloud, w.mu, w.queries)
    assert np.all(normwise(y, ref) <= TOL)
    assert np.array_equal(c.astype(np.int64), rc)


@pytest.mark.parametrize("beta", [0.5, 1.0, 2.0, 4.0])
def test_scene_betas(beta):
    w = syn.workload("scene-200k", scale=0.1)
    y, ref, c, rc = _run(w.cloud, w.mu, w.queries[:30011], beta)
    assert np.all(normwise(y, ref) <= TOL), normwise(y, ref)
    assert np.array_equal(c.astype(np.int64), rc)


@pytest.mark.parametrize("C", [1, 2, 3, 5, 8, 16, 20, 33, 36, 40, 64])
def test_channel_counts(C):
    w = syn.workload("scene-200k", scale=0.05)
    mu = syn.attributes(w.cloud.n, C, seed=C)
    y, ref, _, _ = _run(w.cloud, mu, w.queries[:5000], counts=False)
    assert y.shape == (5000, C)
    assert np.all(normwise(y, ref) <= TOL)


@pytest.mark.parametrize("leaf_size", [1, 4, 16])
def test_leaf_sizes(leaf_size):
    w = syn.workload("scene-200k", scale=0.05)
    y, ref, c, rc = _run(w.cloud, w.mu, w.queries[:7000], leaf_size=leaf_size)
    assert np.all(normwise(y, ref) <= TOL)
    assert np.array_equal(c.astype(np.int64), rc)


def test_no_far_node_is_brute_force():
    """beta -> infinity opens every node: the GPU sum is exact, compared with the
    oracle's brute force (the plain definition, eq. dipole_sum)."""
    w = syn.workload("sphere-2k")
    c = w.cloud
    y, _, _, _ = _run(c, w.mu, w.queries, beta=1e30, counts=False)
    bf = oracle.brute_forward(c.points, c.normals, c.areas, c.eps, w.mu, w.queries)
    assert np.all(normwise(y, bf) <= TOL)


def test_singular_kernel_eps_zero_and_queries_on_points():
    """eps = 0 (eq. pcwn) and queries exactly at points (a zero-distance term is 0)."""
    cl = syn.sphere_cloud(3000, seed=4, eps=None)
    mu = syn.attributes(cl.n, 2, seed=5, kind="unit01")
    q = np.concatenate([cl.points[:64], syn.uniform_box_queries(1000, seed=6)])
    y, ref, c, rc = _run(cl, mu, q)
    assert np.all(np.isfinite(y))
    assert np.all(normwise(y, ref) <= TOL)
    assert np.array_equal(c.astype(np.int64), rc)


def test_small_and_ragged_sizes():
    rng = np.random.default_rng(11)
    for n in [1, 2, 9, 70]:
        p = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
        cl = syn.Cloud(p, syn._unit(rng.normal(size=(n, 3))).astype(np.float32),
                       rng.uniform(0.01, 0.1, n).astype(np.float32),
                       rng.uniform(0.0, 0.2, n).astype(np.float32))
        mu = rng.normal(size=(n, 3)).astype(np.float32)
        for nq in [1, 31, 33, 65]:
            q = rng.uniform(-2, 2, (nq, 3)).astype(np.float32)
            y, ref, c, rc = _run(cl, mu, q)
            assert np.all(normwise(y, ref) <= TOL), (n, nq)
            assert np.array_equal(c.astype(np.int64), rc)


def test_duplicate_points_deep_leaf():
    """Many coincident points: a depth-10 leaf with more than leaf_size points."""
    rng = np.random.default_rng(12)
    p = np.concatenate([np.zeros((50, 3)), rng.uniform(-1, 1, (500, 3))]).astype(np.float32)
    n = len(p)
    cl = syn.Cloud(p, syn._unit(rng.normal(size=(n, 3))).astype(np.float32),
                   np.full(n, 0.01, np.float32), np.full(n, 0.03, np.float32))
    mu = rng.uniform(0, 1, (n, 1)).astype(np.float32)
    q = np.concatenate([rng.normal(scale=0.05, size=(300, 3)),
                        rng.uniform(-1, 1, (300, 3))]).astype(np.float32)
    y, ref, c, rc = _run(cl, mu, q)
    assert np.all(normwise(y, ref) <= TOL)
    assert np.array_equal(c.astype(np.int64), rc)


def test_zero_queries_and_state_errors():
    import torch
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("sphere-2k")
    gt = gpu_tree(w.cloud)
    with pytest.raises(dipole.DipoleError) as e:
        gt.forward(to_dev(w.queries[:10]), 2.0)
    assert e.value.code == dipole.DIPOLE_ESTATE
    gt.refit(to_dev(w.mu))
    out = gt.forward(torch.zeros((0, 3), device="cuda"), 2.0)
    assert out.shape == (0, 1)
    with pytest.raises(dipole.DipoleError):
        gt.forward(to_dev(w.queries[:10]), 0.0)
    gt.sync_status()


def test_nonfinite_query_is_reported_not_hung():
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("sphere-2k")
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    q = w.queries[:100].copy()
    q[7, 0] = np.nan
    y = gt.forward(to_dev(q), 2.0).cpu().numpy()
    with pytest.raises(dipole.DipoleError) as e:
        gt.sync_status()
    assert e.value.code == dipole.DIPOLE_ENONFINITE
    ref = oracle_tree(w.cloud)
    ref.update(w.mu)
    r = ref.forward(np.delete(q, 7, axis=0), 2.0)
    assert np.all(normwise(np.delete(y, 7, axis=0), r) <= TOL)
    gt.sync_status()  # cleared


def test_bf16_attributes():
    """Attributes stored as bfloat16.  The kernel's own error, against the
    oracle on the same bf16-rounded attributes, is gated at 1e-4 (max norm per
    channel).  The error against the float32 attributes is gated at 3e-3 as the
    max-norm relative error of each channel (the error metric of the float
    path, applied to the bf16 path's tolerance).  On zero-mean N(0,1) feature
    channels the bf16 rounding of the inputs alone (the oracle on rounded
    against unrounded attributes, no GPU involved) can exceed 3e-3; there the
    gate cannot be met by any implementation that stores the attributes in
    bf16, and the test reports it as an expected failure with the figures."""
    import torch
    w = syn.workload("scene-200k", scale=0.1)
    mu = syn.attributes(w.cloud.n, 16, seed=21)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(mu).to(torch.bfloat16))
    q = w.queries[:20000]
    y = gt.forward(to_dev(q), 2.0).cpu().numpy()
    ot = oracle_tree(w.cloud)
    ot.update(bf16_round(mu))
    ref_b = ot.forward(q, 2.0)
    assert np.all(normwise(y, ref_b) <= TOL), normwise(y, ref_b)
    ot.update(mu)
    ref = ot.forward(q, 2.0)
    _bf16_gate(normwise(y, ref), normwise(ref_b, ref))


@pytest.mark.parametrize("C,G", [(1, 1), (2, 2), (4, 4), (16, 16), (33, 33), (6, 2), (33, 1)])
def test_bf16_moments(C, G):
    """DIPOLE_BF16_MOMENTS: the value forward reads the node moments rounded to
    bf16.  Against the oracle with the same rounding (reading R13) on the same
    bf16-rounded attributes: 1e-4 per channel, plain and planned (ranged)
    walks, decisions unchanged; an element may differ in addition by the
    oracle's allowance for sums on the edge of a bf16 rounding boundary (the
    GPU sums a leaf in float, the oracle in double); against the float32 attributes and double
    moments the 3e-3 gate of the bf16 path, as in test_bf16_attributes."""
    import torch
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("scene-200k", scale=0.1)
    mu = syn.attributes(w.cloud.n, C, seed=30 + C)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(mu).to(torch.bfloat16), bf16_moments=True,
             geometry_channels=None if G == C else G)
    assert dipole.dipole_tree_info_get(gt.handle)["dtype"] == dipole.DIPOLE_BF16_MOMENTS
    q = w.queries[:20000]
    X = to_dev(q)
    y = gt.forward(X, 2.0).cpu().numpy()
    plan = dipole.QueryPlan(len(q), X.device)
    yp = gt.forward(X, 2.0, plan=plan).cpu().numpy()
    cnt = gt.query_counts(X, 2.0).cpu().numpy()
    gt.sync_status()
    ot = oracle_tree(w.cloud)
    ot.update(bf16_round(mu), geometry_channels=G, bf16_moments=True)
    ref_m, allow = ot.forward_bf16_allowance(q, 2.0)
    _, rc = ot.forward(q, 2.0, counters=True)
    assert np.all(excess_over_allowance(y, ref_m, allow) <= TOL)
    assert np.all(excess_over_allowance(yp, ref_m, allow) <= TOL)
    assert np.array_equal(cnt.astype(np.int64), rc)
    ot.update(mu, geometry_channels=G)
    ref = ot.forward(q, 2.0)
    _bf16_gate(normwise(y, ref), normwise(ref_m, ref))


def _bf16_gate(err, quant, gate=3e-3):
    """err: the GPU's max-norm error against the float32 attributes per
    channel; quant: that of the bf16-rounded inputs alone (oracle vs oracle)."""
    ok = quant <= gate
    assert np.all(err[ok] <= gate), (err, quant)
    if not np.all(ok):
        bad = np.flatnonzero(~ok)
        pytest.xfail(f"3e-3 max-norm gate not met on channels {bad.tolist()}: bf16 rounding of "
                     f"the inputs alone gives {np.round(quant[bad], 5).tolist()}, the GPU "
                     f"{np.round(err[bad], 5).tolist()}")


@pytest.mark.slow
def test_full_size_scene_1m_sampled():
    """The benchmark's workload and launch configuration (1M points, 524,288
    ray-sample queries, C = 4): all queries on the GPU, 4096 sampled ones
    checked against the oracle, decisions bit-exact."""
    w = syn.workload("scene-1m")
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    q = to_dev(w.queries)
    y = gt.forward(q, 2.0).cpu().numpy()
    cnt = gt.query_counts(q, 2.0).cpu().numpy()
    gt.sync_status()
    idx = np.random.default_rng(0).choice(len(w.queries), 4096, replace=False)
    ot = oracle_tree(w.cloud)
    ot.update(w.mu)
    ref, rc = ot.forward(w.queries[idx], 2.0, counters=True)
    assert np.all(normwise(y[idx], ref) <= TOL), normwise(y[idx], ref)
    assert np.array_equal(cnt[idx].astype(np.int64), rc)


def test_ranged_walk_edge_cases():
    """Above 65,536 queries every packet's walk runs as two ranged items: a tree
    that is a single leaf (no cut inside the walk) and 70,000 identical queries
    (an empty code range) still give the exact sums, forward and adjoint."""
    import torch
    cl = syn.sphere_cloud(5, seed=11, eps=0.05)
    mu = syn.attributes(cl.n, 4, seed=12)
    q = syn.uniform_box_queries(70000, seed=13)
    y, ref, c, rc = _run(cl, mu, q)
    assert np.all(normwise(y, ref) <= TOL)
    assert np.array_equal(c.astype(np.int64), rc)
    w = syn.workload("scene-200k", scale=0.05)
    same = np.repeat(w.queries[100:101], 70000, axis=0)
    y2, ref2, _, _ = _run(w.cloud, w.mu, same, counts=False)
    assert np.all(normwise(y2, ref2) <= TOL)
    assert np.all(y2 == y2[0])  # every copy takes the same two-part sum
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    g = syn.upstream_grad(70000, 4, seed=14)
    ga = gt.adjoint(to_dev(same), 2.0, to_dev(g)).cpu().numpy()
    gt.sync_status()
    ot = oracle_tree(w.cloud)
    ot.update(w.mu)
    ref_a = ot.adjoint(w.queries[100:101], 2.0, g.astype(np.float64).sum(0, keepdims=True))
    assert np.all(normwise(ga, ref_a) <= 1e-3)


def test_big_path_outside_queries_and_repeatability():
    """The two-item path (>= 65,536 queries, Hilbert-ordered packets, cost
    buckets) with a ragged count, a fifth of the queries far outside the
    tree's cube (clamped to its border cells by the sort key only), matches
    the oracle; two calls give bitwise the same sums."""
    w = syn.workload("scene-200k", scale=0.05)
    rng = np.random.default_rng(21)
    q = syn.uniform_box_queries(70001, seed=22)
    far = rng.random(len(q)) < 0.2
    q[far] *= np.float32(40.0)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    qd = to_dev(q)
    y1 = gt.forward(qd, 2.0).cpu().numpy()
    y2 = gt.forward(qd, 2.0).cpu().numpy()
    gt.sync_status()
    assert np.array_equal(y1.view(np.uint32), y2.view(np.uint32))
    ot = oracle_tree(w.cloud)
    ot.update(w.mu)
    ref = ot.forward(q, 2.0)
    assert np.all(normwise(y1, ref) <= TOL)


def test_decisions_at_the_far_test_boundary():
    """Queries placed on the boundary spheres |x - p~| = beta r~ of many nodes (in
    float, some land exactly on it, where the strict test opens the node): the
    GPU takes the oracle's decisions (per-query counts bit-exact) and its sums
    match (1e-4); the oracle's near-tie diagnostic sees them."""
    w = syn.workload("scene-200k", scale=0.05)
    ot = oracle_tree(w.cloud)
    ot.update(w.mu)
    ex = ot.export()
    rng = np.random.default_rng(17)
    inner = np.flatnonzero(ex["is_leaf"] == 0)
    t = rng.choice(inner, 3000)
    u = rng.normal(size=(3000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    q = (ex["cen32"][t].astype(np.float64) + 2.0 * ex["r32"][t, None].astype(np.float64) * u).astype(np.float32)
    assert ot.near_ties(q, 2.0).sum() >= 1000
    y, ref, c, rc = _run(w.cloud, w.mu, q)
    assert np.all(normwise(y, ref) <= TOL)
    assert np.array_equal(c.astype(np.int64), rc)
