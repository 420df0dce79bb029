"""GPU appearance channels without the foreshortening term (the oracle's reading
R12; dipole_refit_appearance) against the oracle's FP64 Barnes-Hut on the same
tree: forward 1e-4, adjoint 1e-3 per channel (max norm), decisions bit-exact
(the walk is the same), mixed channel layouts, bf16 attributes, the ranged and
plain walks, the dense grid and the no-allocation forward; gradient entry
points refuse such trees."""
import ctypes

import numpy as np
import pytest

from paper_2405_16788_gb300 import synthetic as syn
from _helpers import bf16_round, gpu_tree, normwise, oracle_tree, to_dev

pytestmark = pytest.mark.gpu


def _setup(C, G, nq, dtype="f32", scale=0.1, seed=41):
    import torch
    w = syn.workload("scene-200k", scale=scale)
    mu = syn.attributes(w.cloud.n, C, seed=seed)
    q = w.queries[:nq]
    gt = gpu_tree(w.cloud)
    m = to_dev(mu) if dtype == "f32" else to_dev(mu).to(torch.bfloat16)
    gt.refit(m, geometry_channels=G)
    ot = oracle_tree(w.cloud)
    ot.update(mu if dtype == "f32" else bf16_round(mu), geometry_channels=G)
    return w, mu, q, gt, ot


@pytest.mark.parametrize("C,G,nq", [(4, 1, 3001), (4, 1, None), (4, 0, 20000), (3, 2, 9000),
                                    (16, 4, 20000), (33, 1, 5000)])
def test_forward_and_adjoint_match_oracle(C, G, nq):
    w, mu, q, gt, ot = _setup(C, G, nq)
    X = to_dev(q)
    y = gt.forward(X, 2.0).cpu().numpy()
    g = syn.upstream_grad(len(q), C, seed=C + G)
    ga = gt.adjoint(X, 2.0, to_dev(g)).cpu().numpy()
    cnt = gt.query_counts(X, 2.0).cpu().numpy()
    gt.sync_status()
    idx = np.arange(len(q)) if len(q) <= 20000 else np.random.default_rng(2).choice(len(q), 20000, replace=False)
    ref, rc = ot.forward(q[idx], 2.0, counters=True)
    assert np.all(normwise(y[idx], ref) <= 1e-4), normwise(y[idx], ref)
    assert np.array_equal(cnt[idx].astype(np.int64), rc)
    if len(idx) == len(q):
        aref = ot.adjoint(q, 2.0, g.astype(np.float64))
        assert np.all(normwise(ga, aref) <= 1e-3), normwise(ga, aref)


def test_planned_adjoint_and_bf16():
    import torch
    from paper_2405_16788_gb300 import dipole
    w, mu, q, gt, ot = _setup(4, 1, None, dtype="bf16")
    X = to_dev(q)
    plan = dipole.QueryPlan(len(q), X.device)
    y = gt.forward(X, 2.0, plan=plan).cpu().numpy()
    idx = np.random.default_rng(3).choice(len(q), 3000, replace=False)
    g = np.zeros((len(q), 4), np.float32)
    g[idx] = syn.upstream_grad(3000, 4, seed=5)
    ga = gt.adjoint(X, 2.0, to_dev(g), plan=plan).cpu().numpy()
    gt.sync_status()
    assert np.all(normwise(y[idx], ot.forward(q[idx], 2.0)) <= 1e-4)
    aref = ot.adjoint(q[idx], 2.0, g[idx].astype(np.float64))
    assert np.all(normwise(ga, aref) <= 1e-3), normwise(ga, aref)


def test_grid_noalloc_and_moments():
    import torch
    from paper_2405_16788_gb300 import dipole
    w, mu, q, gt, ot = _setup(4, 1, 4000)
    lo, h, dims = (-1.2, -1.1, -1.0), 0.1, (17, 13, 11)
    grid = gt.forward_grid(lo, h, dims, 2.0).cpu().numpy().reshape(-1, 4)
    ax = [np.float32(lo[d]) + np.arange(dims[d]).astype(np.float32) * np.float32(h) for d in range(3)]
    z, yy, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    pts = np.stack([x, yy, z], -1).reshape(-1, 3).astype(np.float32)
    assert np.all(normwise(grid, ot.forward(pts, 2.0)) <= 1e-4)
    out = torch.empty((len(q), 4), device="cuda")
    dipole.dipole_forward_noalloc(gt.handle, to_dev(q), 2.0, out)
    assert np.all(normwise(out.cpu().numpy(), ot.forward(q, 2.0)) <= 1e-4)
    ex = gt.export(moments=True)
    M = ex["moments"].reshape(-1, 4, 3)
    assert np.all(M[:, 1:, 1:] == 0.0)  # appearance channels: M in the first slot only
    # root: M^c = sum A mu^c, S^0 = sum A n mu^0 (float sums against double)
    c = w.cloud
    Mref = (c.areas[:, None].astype(np.float64) * mu[:, 1:]).sum(0)
    assert np.allclose(M[0, 1:, 0], Mref, rtol=1e-5, atol=1e-6 * np.abs(Mref).max())
    Sref = ((c.areas[:, None] * c.normals).astype(np.float64) * mu[:, :1]).sum(0)
    assert np.allclose(M[0, 0], Sref, rtol=1e-4, atol=1e-6 * np.abs(Sref).max())
    gt.sync_status()


def test_gradient_entry_points_refuse_appearance_channels():
    from paper_2405_16788_gb300 import dipole
    w, mu, q, gt, ot = _setup(4, 1, 100)
    X = to_dev(q)
    with pytest.raises(dipole.DipoleError) as e:
        gt.forward_grad(X, 2.0)
    assert e.value.code == dipole.DIPOLE_EINVAL
    with pytest.raises(dipole.DipoleError):
        gt.adjoint_queries(X, 2.0, to_dev(np.ones((100, 4), np.float32)))
    with pytest.raises(dipole.DipoleError):
        gt.adjoint_geom(X, 2.0, to_dev(np.ones((100, 4), np.float32)))
    # a plain refit restores them
    gt.refit(to_dev(mu))
    gt.forward_grad(X, 2.0)
    gt.sync_status()
