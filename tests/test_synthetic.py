"""The seeded input recipe: every workload is reproducible from its seeds and
has the sizes, value ranges and structure its description states (the same
inputs feed the CUDA path and the oracle)."""
import math

import numpy as np
import pytest

from paper_2405_16788_gb300 import synthetic as syn


def _same(a, b):
    return a.dtype == b.dtype and a.shape == b.shape and np.array_equal(a, b)


@pytest.mark.parametrize("name,scale", [("sphere-2k", 1.0), ("scene-200k", 0.05),
                                        ("scene-1m", 0.02), ("scene-5m-loop", 0.002)])
def test_workloads_are_reproducible(name, scale):
    a, b = syn.workload(name, scale), syn.workload(name, scale)
    for x, y in [(a.cloud.points, b.cloud.points), (a.cloud.normals, b.cloud.normals),
                 (a.cloud.areas, b.cloud.areas), (a.mu, b.mu), (a.queries, b.queries)]:
        assert _same(x, y)
    assert (a.cloud.eps is None) == (b.cloud.eps is None)
    if a.cloud.eps is not None:
        assert _same(a.cloud.eps, b.cloud.eps)


def test_sphere_2k_recipe():
    w = syn.workload("sphere-2k")
    c = w.cloud
    assert c.n == 2000 and w.queries.shape == (4096, 3) and w.mu.shape == (2000, 1)
    assert np.allclose(np.linalg.norm(c.points.astype(np.float64), axis=1), 1.0, atol=1e-6)
    assert np.allclose(c.normals, c.points, atol=1e-6)  # outward unit normals
    assert math.isclose(float(c.areas.astype(np.float64).sum()), 4 * math.pi, rel_tol=1e-5)
    assert np.all(c.eps == np.float32(0.02))
    assert np.all(np.abs(w.queries) <= 1.5) and w.mu.min() >= 0.0 and w.mu.max() <= 1.0


def test_scene_recipe_full_size():
    w = syn.workload("scene-1m")
    c = w.cloud
    assert c.n == 1_000_000 and w.queries.shape == (524_288, 3) and w.mu.shape == (1_000_000, 4)
    for a in (c.points, c.normals, c.areas, c.eps, w.mu, w.queries):
        assert a.dtype == np.float32 and np.all(np.isfinite(a))
    assert np.allclose(np.linalg.norm(c.normals.astype(np.float64), axis=1), 1.0, atol=1e-5)
    assert np.all(c.areas > 0)
    assert c.eps.min() >= np.float32(0.002) * (1 - 1e-6) and c.eps.max() <= np.float32(0.02) * (1 + 1e-6)
    # log-uniform radii: the median sits near the geometric mean of the range
    assert abs(math.log(float(np.median(c.eps))) - 0.5 * math.log(0.002 * 0.02)) < 0.05
    assert c.meta["outliers"] == 20_000
    # channel 0 geometry U(0.5, 1.5), channels 1-3 colour U(0, 1)
    assert 0.5 <= w.mu[:, 0].min() and w.mu[:, 0].max() <= 1.5
    assert 0.0 <= w.mu[:, 1:].min() and w.mu[:, 1:].max() <= 1.0
    # the queries are ray samples clipped to the sphere of radius 1.5
    assert np.linalg.norm(w.queries.astype(np.float64), axis=1).max() <= 1.5 + 1e-5
    # inliers lie near the torus (R = 0.6, r = 0.2) or the spheres (0.3 at z = +-0.55)
    p = c.points.astype(np.float64)
    d_torus = np.abs(np.hypot(np.hypot(p[:, 0], p[:, 1]) - 0.6, p[:, 2]) - 0.2)
    d_sph = np.minimum(np.abs(np.linalg.norm(p - [0, 0, 0.55], axis=1) - 0.3),
                       np.abs(np.linalg.norm(p - [0, 0, -0.55], axis=1) - 0.3))
    near = np.minimum(d_torus, d_sph) < 0.03  # 6 sigma of the 0.005 noise
    assert abs(int(near.sum()) - 980_000) < 2_000  # inliers, and a few outliers that land close


def test_scene_input_order_has_no_spatial_structure():
    c = syn.workload("scene-200k", 0.05).cloud
    step = np.linalg.norm(np.diff(c.points.astype(np.float64), axis=0), axis=1)
    assert np.median(step) > 0.3  # consecutive points are far apart: a shuffled cloud


def test_attributes_channel_kinds():
    mu = syn.attributes(10_000, 16, seed=7)
    assert mu.shape == (10_000, 16)
    feat = mu[:, 4:].astype(np.float64)
    assert abs(feat.mean()) < 0.02 and abs(feat.std() - 1.0) < 0.02
    u = syn.attributes(1000, 3, seed=7, kind="unit01")
    assert u.min() >= 0.0 and u.max() <= 1.0
    g = syn.upstream_grad(1000, 3, seed=1)
    assert g.shape == (1000, 3) and g.dtype == np.float32
