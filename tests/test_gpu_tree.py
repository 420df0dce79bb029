"""GPU tree construction vs the oracle: every integer array bit-exact, and the
float node geometry that the far test reads (centroid, radius) bit-exact too,
because both sides follow the same specified operation order."""
import numpy as np
import pytest

from paper_2405_16788_gb300 import synthetic as syn
from _helpers import gpu_tree, oracle_tree

pytestmark = pytest.mark.gpu

INT_KEYS = ["code", "perm", "first", "count", "level", "parent", "skip", "is_leaf"]


def _compare(cloud, leaf_size=8, max_depth=10):
    g = gpu_tree(cloud, leaf_size, max_depth).export()
    o = oracle_tree(cloud, leaf_size, max_depth).export()
    for k in INT_KEYS:
        assert np.array_equal(g[k].astype(np.int64), o[k].astype(np.int64)), k
    assert np.array_equal(g["cen32"], o["cen32"])
    assert np.array_equal(g["r32"], o["r32"])
    assert np.array_equal(g["area"], o["area"])
    assert np.array_equal(g["eps"], o["eps"].astype(np.float32))
    return g


def _tiny_clouds():
    rng = np.random.default_rng(3)
    out = []
    for n in [1, 2, 7, 8, 9, 31, 33, 100]:
        p = rng.uniform(-1, 1, (n, 3))
        out.append(p)
    base = rng.uniform(-1, 1, (4, 3))
    out.append(base[rng.integers(0, 4, 200)])              # heavy duplicates
    out.append(np.zeros((40, 3)))                           # all points equal
    out.append(np.concatenate([rng.normal(scale=1e-5, size=(50, 3)), [[3.0, -2, 1]]]))
    clouds = []
    for p in out:
        n = len(p)
        nr = syn._unit(rng.normal(size=(n, 3)))
        a = rng.uniform(0.01, 0.1, n)
        e = rng.uniform(0.0, 0.05, n)
        clouds.append(syn.Cloud(p.astype(np.float32), nr.astype(np.float32),
                                a.astype(np.float32), e.astype(np.float32)))
    return clouds


@pytest.mark.parametrize("leaf_size,max_depth", [(8, 10), (1, 10), (3, 10), (8, 4), (5, 0)])
def test_tree_bit_exact_small(leaf_size, max_depth):
    for cl in _tiny_clouds():
        _compare(cl, leaf_size, max_depth)


def test_tree_bit_exact_sphere():
    _compare(syn.workload("sphere-2k").cloud)


def test_tree_bit_exact_scene_200k():
    g = _compare(syn.workload("scene-200k").cloud)
    assert g["is_leaf"].sum() > 10000


def test_tree_bit_exact_scene_1m():
    """The full 1M-point cloud of the benchmark workload."""
    _compare(syn.workload("scene-1m").cloud)


def test_build_rejects_bad_inputs():
    import torch
    from paper_2405_16788_gb300 import dipole
    cl = syn.workload("sphere-2k").cloud
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bad_a = cl.areas.copy()
    bad_a[17] = 0.0
    with pytest.raises(dipole.DipoleError) as e:
        dipole.DipoleTree(t(cl.points), t(cl.normals), t(bad_a), t(cl.eps))
    assert e.value.code == dipole.DIPOLE_EINVAL
    bad_p = cl.points.copy()
    bad_p[5, 1] = np.nan
    with pytest.raises(dipole.DipoleError) as e:
        dipole.DipoleTree(t(bad_p), t(cl.normals), t(cl.areas), t(cl.eps))
    assert e.value.code == dipole.DIPOLE_ENONFINITE
    bad_e = cl.eps.copy()
    bad_e[3] = -1.0
    with pytest.raises(dipole.DipoleError) as e:
        dipole.DipoleTree(t(cl.points), t(cl.normals), t(cl.areas), t(bad_e))
    assert e.value.code == dipole.DIPOLE_EINVAL
    with pytest.raises(dipole.DipoleError):
        dipole.DipoleTree(t(cl.points), t(cl.normals), t(cl.areas), t(cl.eps), leaf_size=0)
    # a good build still works after the failures
    tr = dipole.DipoleTree(t(cl.points), t(cl.normals), t(cl.areas), t(cl.eps))
    assert tr.info["n_points"] == cl.n
