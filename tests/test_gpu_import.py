"""Checkpoint / resume of a tree (dipole_tree_export -> dipole_tree_import) and
failure detection on a corrupt tree: a traversal that cannot finish stops at
its step bound and reports DIPOLE_ETRAVERSAL; the GPU context stays usable.
The corruption is made on the host (a skip index pointing back at its own
node); no fault, trap or endless loop is involved."""
import numpy as np
import pytest

from paper_2405_16788_gb300 import synthetic as syn
from _helpers import to_dev

pytestmark = pytest.mark.gpu


def _inputs(w):
    c = w.cloud
    return to_dev(c.points), to_dev(c.normals), to_dev(c.areas), to_dev(c.eps)


def test_export_import_round_trip_is_exact():
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("scene-200k", scale=0.1)
    P, N, A, E = _inputs(w)
    t0 = dipole.DipoleTree(P, N, A, E)
    ex = t0.export()
    t1 = dipole.DipoleTree.from_export(P, N, A, E, ex)
    ex1 = t1.export()
    for k in ["code", "perm", "first", "count", "level", "parent", "skip", "is_leaf", "cen32",
              "r32", "area", "eps"]:
        assert np.array_equal(ex[k], ex1[k]), k
    mu = to_dev(w.mu)
    q = to_dev(w.queries[:20000])
    t0.refit(mu)
    t1.refit(mu)
    y0 = t0.forward(q, 2.0).cpu().numpy()
    y1 = t1.forward(q, 2.0).cpu().numpy()
    assert np.array_equal(y0, y1)
    g = to_dev(syn.upstream_grad(20000, 4, seed=3))
    a0 = t0.adjoint(q, 2.0, g).cpu().numpy()
    a1 = t1.adjoint(q, 2.0, g).cpu().numpy()
    assert np.allclose(a0, a1, rtol=1e-5, atol=1e-7)  # float atomics: order may differ
    t0.sync_status()
    t1.sync_status()


def test_corrupt_tree_reports_traversal_error_and_context_survives():
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("sphere-2k")
    P, N, A, E = _inputs(w)
    good = dipole.DipoleTree(P, N, A, E)
    ex = good.export()
    bad = {k: v.copy() for k, v in ex.items()}
    leaf = int(np.nonzero(bad["is_leaf"])[0][0])
    bad["skip"][leaf] = leaf  # a leaf whose successor is itself: a cycle
    t = dipole.DipoleTree.from_export(P, N, A, E, bad)
    t.refit(to_dev(w.mu))
    s, k = int(bad["first"][leaf]), int(bad["count"][leaf])
    perm = bad["perm"][s:s + k]
    q = to_dev(w.cloud.points[perm] + 1e-3)  # queries at that leaf's own points
    t.forward(q, 2.0)
    with pytest.raises(dipole.DipoleError) as e:
        t.sync_status()
    assert e.value.code == dipole.DIPOLE_ETRAVERSAL
    # the device and the good tree keep working
    good.refit(to_dev(w.mu))
    y = good.forward(to_dev(w.queries), 2.0)
    good.sync_status()
    assert bool(y.isfinite().all())
