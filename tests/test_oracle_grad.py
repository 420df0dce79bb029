"""Pins for the oracle's spatial gradient of the dipole sum (the oracle's reading R9) and its
adjoint, against finite differences of the plain sum, closed forms and the
adjoint identity."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_16788_gb300 import synthetic as syn


def _fd_grad_brute(c, mu, x, h=1e-5):
    """Central differences of the brute-force sum in float64 queries: the
    queries are passed as float32, so use an h that float32 represents well
    around x and the actual float32 step."""
    out = np.zeros((len(x), mu.shape[1], 3))
    for k in range(3):
        xp = x.astype(np.float64).copy()
        xm = xp.copy()
        xp[:, k] += h
        xm[:, k] -= h
        xp32, xm32 = xp.astype(np.float32), xm.astype(np.float32)
        dp = oracle.brute_forward(c.points, c.normals, c.areas, c.eps, mu, xp32)
        dm = oracle.brute_forward(c.points, c.normals, c.areas, c.eps, mu, xm32)
        step = (xp32[:, k].astype(np.float64) - xm32[:, k].astype(np.float64))[:, None]
        out[:, :, k] = (dp - dm) / step
    return out


def test_brute_gradient_matches_finite_differences():
    w = syn.workload("scene-200k", scale=0.01)
    c = w.cloud
    rng = np.random.default_rng(0)
    # queries near points (small t), at moderate and at large distance
    near = c.points[rng.choice(c.n, 20)] + rng.normal(scale=0.004, size=(20, 3))
    far = rng.uniform(-1.2, 1.2, size=(20, 3))
    x = np.concatenate([near, far]).astype(np.float32)
    g = oracle.brute_forward_grad(c.points, c.normals, c.areas, c.eps, w.mu, x)
    fd = _fd_grad_brute(c, w.mu, x, h=1e-5)
    scale = np.max(np.abs(g), axis=(0, 2))
    err = np.max(np.abs(g - fd), axis=(0, 2)) / scale
    assert np.all(err < 2e-5), err


def test_disk_axis_gradient_closed_form():
    """eps = 0, a disk of radius a with normal +z: on its axis
    dD/dh = (1/2) a^2 / (h^2 + a^2)^(3/2) on both sides, and no radial part."""
    a, nr, nt = 1.0, 300, 600
    r_mid = (np.arange(nr) + 0.5) * a / nr
    th = (np.arange(nt) + 0.5) * 2 * math.pi / nt
    R, TH = np.meshgrid(r_mid, th, indexing="ij")
    pts = np.stack([R * np.cos(TH), R * np.sin(TH), np.zeros_like(R)], -1).reshape(-1, 3)
    area = (R * (a / nr) * (2 * math.pi / nt)).reshape(-1)
    nrm = np.broadcast_to([0.0, 0.0, 1.0], pts.shape)
    hs = np.array([0.4, -0.4, 1.0, -2.5])
    q = np.stack([np.zeros_like(hs), np.zeros_like(hs), hs], -1).astype(np.float32)
    g = oracle.brute_forward_grad(pts, nrm, area, None, np.ones(len(area)), q)[:, 0, :]
    ref = 0.5 * a * a / (hs.astype(np.float32).astype(np.float64) ** 2 + a * a) ** 1.5
    assert np.allclose(g[:, 2], ref, rtol=1e-4)
    assert np.all(np.abs(g[:, :2]) < 1e-6)


def _blurred_ball(s, R, eps):
    a, b = (R - s) / eps, (R + s) / eps
    return 0.5 * (math.erf(a) + math.erf(b)) - eps / (2 * s * math.sqrt(math.pi)) * (
        math.exp(-a * a) - math.exp(-b * b))


def test_sphere_gradient_is_radial_derivative_of_blurred_indicator():
    """Prop. 1: D = W(|x|) for a dense sphere, so grad D = W'(s) x/s (W' by
    central differences of the closed form)."""
    eps, R, n = 0.15, 1.0, 40000
    cl = syn.sphere_cloud(n, seed=0, eps=eps, radius=R, fibonacci=True)
    s_list = [0.3, 0.8, 0.95, 1.05, 1.3]
    dirs = syn._unit(np.random.default_rng(5).normal(size=(len(s_list), 3)))
    q = (np.array(s_list)[:, None] * dirs).astype(np.float32)
    g = oracle.brute_forward_grad(cl.points, cl.normals, cl.areas, cl.eps, np.ones(n), q)[:, 0, :]
    for x, gv in zip(q.astype(np.float64), g):
        s = float(np.linalg.norm(x))
        h = 1e-5
        dw = (_blurred_ball(s + h, R, eps) - _blurred_ball(s - h, R, eps)) / (2 * h)
        assert np.allclose(gv, dw * x / s, atol=5e-4), (s, gv, dw * x / s)


def test_gradient_limit_at_small_distance():
    """As r -> 0 the radial factor a = rho/r^3 -> 4/(3 sqrt(pi) eps^3) (the
    paper's finite value at the origin, Sec. 4.1), so one point's gradient
    tends to -A mu a(0) n / (4 pi)."""
    eps, A = 0.2, 0.7
    nrm = np.array([[0.0, 0.6, 0.8]])
    x = np.array([[1e-4, -2e-4, 1.5e-4]], np.float32)
    g = oracle.brute_forward_grad([[0.0, 0, 0]], nrm, [A], [eps], [1.0], x)[0, 0]
    ref = -A * (4 / (3 * math.sqrt(math.pi) * eps ** 3)) * nrm[0] / (4 * math.pi)
    assert np.allclose(g, ref, rtol=1e-5, atol=1e-9)


def test_bh_gradient_equals_brute_when_nothing_is_far():
    w = syn.workload("sphere-2k", scale=0.5)
    c = w.cloud
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(w.mu)
    a = T.forward_grad(w.queries, np.inf)
    b = oracle.brute_forward_grad(c.points, c.normals, c.areas, c.eps, w.mu, w.queries)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-13)


def test_bh_gradient_matches_finite_differences_of_bh_sum():
    """Where the far decisions do not change between x - h and x + h, the
    Barnes-Hut sum is smooth and its derivative is the Barnes-Hut gradient."""
    w = syn.workload("scene-200k", scale=0.02)
    c = w.cloud
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(w.mu)
    x = w.queries[:400].astype(np.float64)
    h = 3e-5
    g = T.forward_grad(x.astype(np.float32), 2.0)
    _, c0 = T.forward(x.astype(np.float32), 2.0, counters=True)
    checked = 0
    for k in range(3):
        xp, xm = x.copy(), x.copy()
        xp[:, k] += h
        xm[:, k] -= h
        xp32, xm32 = xp.astype(np.float32), xm.astype(np.float32)
        dp, cp = T.forward(xp32, 2.0, counters=True)
        dm, cm = T.forward(xm32, 2.0, counters=True)
        same = np.all(cp == c0, axis=1) & np.all(cm == c0, axis=1)
        step = (xp32[:, k].astype(np.float64) - xm32[:, k].astype(np.float64))
        fd = (dp - dm) / step[:, None]
        scale = np.max(np.abs(g[:, :, k]))
        assert np.all(np.abs(fd[same] - g[same, :, k]) < 2e-4 * scale)
        checked += same.sum()
    assert checked > 600


def test_bh_gradient_adjoint_identity():
    """<g, D> + <G, grad D> = <adjoint(g, G), mu> for Barnes-Hut (linear in mu)."""
    w = syn.workload("scene-200k", scale=0.02)
    c = w.cloud
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(w.mu)
    q = w.queries[:2500]
    D = T.forward(q, 2.0)
    GD = T.forward_grad(q, 2.0)
    g = syn.upstream_grad(len(q), 4, seed=1).astype(np.float64)
    G = np.random.default_rng(2).normal(size=GD.shape)
    dmu = T.adjoint_grad(q, 2.0, g, G)
    lhs = np.sum(g * D) + np.sum(G * GD)
    rhs = np.sum(dmu * w.mu.astype(np.float64))
    assert abs(lhs - rhs) < 1e-10 * (np.sum(np.abs(g * D)) + np.sum(np.abs(G * GD)))
    # the value part alone is the existing adjoint
    assert np.allclose(T.adjoint_grad(q, 2.0, g, None), T.adjoint(q, 2.0, g), rtol=1e-12,
                       atol=1e-15)
