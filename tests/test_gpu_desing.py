"""The desingularized kernel (the oracle's reading R11: 1/max(r, eps)^3, the paper's
ablation baseline) on the GPU against the oracle with the same kernel: forward
1e-4, adjoints 1e-3, decisions bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2405_16788_gb300 import synthetic as syn
from _helpers import normwise, oracle_tree, to_dev

pytestmark = pytest.mark.gpu


def _err(y, ref):
    y = np.asarray(y, np.float64).reshape(len(y), -1)
    ref = np.asarray(ref, np.float64).reshape(len(ref), -1)
    return normwise(y, ref)


def test_desingularized_forward_gradient_and_adjoints():
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("scene-200k", scale=0.05)
    c = w.cloud
    rng = np.random.default_rng(1)
    pick = rng.choice(c.n, 4000)
    near = (c.points[pick] + rng.normal(size=(4000, 3)) * c.eps[pick][:, None]).astype(np.float32)
    q = np.concatenate([w.queries[:16000], near]).astype(np.float32)
    gt = dipole.DipoleTree(to_dev(c.points), to_dev(c.normals), to_dev(c.areas), to_dev(c.eps),
                           kernel="desingularized")
    assert gt.info["kernel"] == dipole.DIPOLE_KERNEL_DESINGULARIZED
    gt.refit(to_dev(w.mu))
    Q = to_dev(q)
    y = gt.forward(Q, 2.0).cpu().numpy()
    cnt = gt.query_counts(Q, 2.0).cpu().numpy()
    d, gx = gt.forward_grad(Q, 2.0)
    g = rng.normal(size=(len(q), 4)).astype(np.float32)
    G = rng.normal(size=(len(q), 4, 3)).astype(np.float32)
    ga = gt.adjoint(Q, 2.0, to_dev(g)).cpu().numpy()
    gm, gn, ge = gt.adjoint_geom(Q, 2.0, to_dev(g), to_dev(G))
    gt.sync_status()
    with oracle.kernel("desingularized"):
        ot = oracle_tree(c)
        ot.update(w.mu)
        ref, rc = ot.forward(q, 2.0, counters=True)
        rgx = ot.forward_grad(q, 2.0)
        rga = ot.adjoint(q, 2.0, g.astype(np.float64))
        rm, rn, re = ot.adjoint_geom(q, 2.0, g.astype(np.float64), G.astype(np.float64))
    assert np.array_equal(cnt.astype(np.int64), rc)
    assert np.all(_err(y, ref) <= 1e-4), _err(y, ref)
    assert np.all(_err(d.cpu().numpy(), ref) <= 1e-4)
    assert np.all(_err(gx.cpu().numpy(), rgx) <= 1e-4), _err(gx.cpu().numpy(), rgx)
    assert np.all(_err(ga, rga) <= 1e-3)
    assert np.all(_err(gm.cpu().numpy(), rm) <= 1e-3)
    assert np.all(_err(gn.cpu().numpy(), rn) <= 1e-3)
    assert np.all(_err(ge.cpu().numpy()[:, None], re[:, None]) <= 1e-3), _err(ge.cpu().numpy()[:, None], re[:, None])
    # and it is not the regularized kernel
    ot2 = oracle_tree(c)
    ot2.update(w.mu)
    assert np.max(_err(y, ot2.forward(q, 2.0))) > 1e-3
