"""Pins of the oracle's appearance channels without the foreshortening term
(reading R12 of oracle/dipole_oracle.c: the paper skips the cosine
n.(p - x)/|p - x| of the kernel for its appearance attributes, Sec. 5.3,
eq. appearance_features).  Without it a point contributes
A rho(r/eps)/(4 pi r^2) mu, a far node A~ rho(d/eps~)/(4 pi d^2) m~ with m~ the
area-weighted mean attribute.

* Closed form: for a uniform sphere of radius R, (1/4 pi) int dA/|x - y|^2 =
  (R / 2s) ln |(R + s)/(R - s)| at distance s from the centre (1 at the centre),
  reproduced by a dense Fibonacci sampling with mu = 1 (a cosine left in, a
  wrong power of r or a dropped 1/(4 pi) is off by orders of magnitude).
* Barnes-Hut equals the plain sum when nothing is far; its error falls as
  beta grows; a far node holding one point is that point's exact term.
* Channels are independent: with G = 1 the first channel equals the dipole sum
  and the others equal the sums without the foreshortening term.
* The adjoint is the transpose: <g, K mu> = <K^T g, mu> for the Barnes-Hut
  operator with mixed channels, and equals the plain adjoint at large beta."""
import numpy as np
import pytest

import oracle
from paper_2405_16788_gb300 import synthetic as syn


def _fib_sphere(N, R=1.0):
    i = np.arange(N) + 0.5
    phi = np.arccos(1 - 2 * i / N)
    th = np.pi * (1 + 5 ** 0.5) * i
    p = R * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    return p.astype(np.float32), np.full(N, 4 * np.pi * R * R / N, np.float32)


@pytest.mark.parametrize("s", [0.0, 0.3, 0.6, 1.5, 2.5, 5.0])
def test_sphere_closed_form(s):
    p, A = _fib_sphere(20000)
    eps = np.full(len(p), 1e-4, np.float32)
    mu = np.ones((len(p), 1), np.float32)
    x = np.array([[0.3 * s, 0.4 * s, np.sqrt(0.75) * s]], np.float32)
    sv = float(np.linalg.norm(x.astype(np.float64)))
    v = oracle.brute_forward_app(p, p, A, eps, mu, x, 0)[0, 0]
    ref = 1.0 if sv == 0 else np.log((1 + sv) / abs(1 - sv)) / (2 * sv)
    assert abs(v - ref) <= 1e-5 * ref, (v, ref)


def _case(C=3, seed=0):
    w = syn.workload("scene-200k", scale=0.02)
    mu = syn.attributes(w.cloud.n, C, seed=seed)
    return w.cloud, mu, w.queries[:600]


def test_bh_equals_plain_sum_when_nothing_is_far_and_converges():
    c, mu, q = _case()
    ref = oracle.brute_forward_app(c.points, c.normals, c.areas, c.eps, mu, q, 1)
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(mu, geometry_channels=1)
    den = np.abs(ref).max(0)
    # nothing far: a node is only far when its radius is 0 (one point, or
    # coincident points), whose far term is the point's own term up to the
    # float rounding of the node centroid (reading R7)
    assert np.all(np.abs(T.forward(q, 1e7) - ref).max(0) / den <= 1e-6)
    errs = [np.abs(T.forward(q, b) - ref).max() / den.max() for b in (1.0, 2.0, 4.0, 8.0)]
    assert all(a > b for a, b in zip(errs, errs[1:])) and errs[-1] < 0.01 * errs[0], errs


def test_single_point_far_node_is_exact():
    p = np.array([[0.0, 0.0, 0.0], [0.5, 0.1, -0.2]], np.float32)
    n = np.array([[0, 0, 1], [1, 0, 0]], np.float32)
    A = np.array([0.3, 0.7], np.float32)
    eps = np.array([0.05, 0.1], np.float32)
    mu = np.array([[1.5, -2.0], [0.25, 3.0]], np.float32)
    q = np.array([[3.0, 2.0, 1.0], [-2.0, 0.5, 4.0]], np.float32)
    T = oracle.Tree(p, n, A, eps, leaf_size=1)
    T.update(mu, geometry_channels=0)
    # beta = 100: the root (two points) is opened, each single-point leaf
    # (radius 0) is far
    got, cnt = T.forward(q, 100.0, counters=True)
    assert np.all(cnt[:, 1] == 2)
    ref = oracle.brute_forward_app(p, n, A, eps, mu, q, 0)
    assert np.allclose(got, ref, rtol=1e-6, atol=0)


def test_channels_are_independent():
    c, mu, q = _case(C=1)
    mu2 = np.repeat(mu, 3, axis=1)
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(mu2, geometry_channels=1)
    mixed = T.forward(q, 2.0)
    T.update(mu, geometry_channels=1)
    dip = T.forward(q, 2.0)
    T.update(mu, geometry_channels=0)
    app = T.forward(q, 2.0)
    assert np.array_equal(mixed[:, 0], dip[:, 0])
    assert np.array_equal(mixed[:, 1], app[:, 0]) and np.array_equal(mixed[:, 2], app[:, 0])
    assert not np.allclose(dip, app)


def test_adjoint_is_the_transpose():
    c, mu, q = _case(C=4, seed=3)
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(mu, geometry_channels=2)
    g = np.random.default_rng(1).normal(size=(len(q), 4))
    lhs = np.sum(g * T.forward(q, 2.0))
    rhs = np.sum(T.adjoint(q, 2.0, g) * mu.astype(np.float64))
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + 1e-300)
    # large beta: the plain adjoint (transpose of the plain sum)
    ref = oracle.brute_adjoint_app(c.points, c.normals, c.areas, c.eps, q, g, 2)
    got = T.adjoint(q, 1e7, g)
    assert np.all(np.abs(got - ref).max(0) / np.abs(ref).max(0) <= 1e-6)


def test_gradients_refuse_appearance_channels():
    c, mu, q = _case()
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(mu, geometry_channels=1)
    with pytest.raises(NotImplementedError):
        T.forward_grad(q, 2.0)
