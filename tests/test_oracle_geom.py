"""Pins for the oracle's gradients with respect to the normals and the
regularization radii (the oracle's reading R10): central differences of the plain sum and
of the Barnes-Hut sum (whose far decisions do not depend on n or eps), the
linearity of D in the normals and in mu, and the eps-derivative of the
closed-form blurred ball indicator (Prop. 1)."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_16788_gb300 import synthetic as syn


def _loss_brute(c, mu, x, g, G, normals=None, eps=None):
    nr = c.normals if normals is None else normals
    e = c.eps if eps is None else eps
    D = oracle.brute_forward(c.points, nr, c.areas, e, mu, x)
    GD = oracle.brute_forward_grad(c.points, nr, c.areas, e, mu, x)
    return np.sum(g * D) + np.sum(G * GD)


def _step(v, h):
    """float32 values v + h and v - h and the actual float32 step between them."""
    vp, vm = np.float32(v + h), np.float32(v - h)
    return vp, vm, float(np.float64(vp) - np.float64(vm))


def _small_case(seed=0, n_q=60):
    w = syn.workload("scene-200k", scale=0.004)
    c = w.cloud
    rng = np.random.default_rng(seed)
    near = c.points[rng.choice(c.n, n_q // 2)] + rng.normal(scale=0.01, size=(n_q // 2, 3))
    far = rng.uniform(-1.2, 1.2, size=(n_q - n_q // 2, 3))
    x = np.concatenate([near, far]).astype(np.float32)
    g = rng.normal(size=(n_q, w.mu.shape[1]))
    G = rng.normal(size=(n_q, w.mu.shape[1], 3))
    return w, c, x, g, G


def test_brute_normal_and_eps_gradients_match_central_differences():
    w, c, x, g, G = _small_case()
    dmu, dn, deps = oracle.brute_adjoint_geom(c.points, c.normals, c.areas, c.eps, w.mu, x, g, G)
    rng = np.random.default_rng(3)
    # points near the queries have large gradients: check those and random ones
    picks = list(rng.choice(c.n, 6, replace=False)) + list(np.argsort(-np.abs(deps))[:4])
    for m in picks:
        for k in range(3):
            nrm = c.normals.astype(np.float32).copy()
            vp, vm, st = _step(nrm[m, k], 1e-3)
            nrm[m, k] = vp
            lp = _loss_brute(c, w.mu, x, g, G, normals=nrm)
            nrm[m, k] = vm
            lm = _loss_brute(c, w.mu, x, g, G, normals=nrm)
            # L is linear in n: central differences are exact up to rounding
            assert abs((lp - lm) / st - dn[m, k]) <= 1e-7 * (1 + abs(dn[m, k])), (m, k)
        e = c.eps.astype(np.float32).copy()
        vp, vm, st = _step(e[m], 1e-4 * e[m])
        e[m] = vp
        lp = _loss_brute(c, w.mu, x, g, G, eps=e)
        e[m] = vm
        lm = _loss_brute(c, w.mu, x, g, G, eps=e)
        fd = (lp - lm) / st
        assert abs(fd - deps[m]) <= 1e-5 * abs(deps[m]) + 1e-9, (m, fd, deps[m])


def test_bh_geom_gradients_equal_brute_when_nothing_is_far():
    w, c, x, g, G = _small_case(seed=1)
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(w.mu)
    a = T.adjoint_geom(x, np.inf, g, G)
    b = oracle.brute_adjoint_geom(c.points, c.normals, c.areas, c.eps, w.mu, x, g, G)
    for u, v in zip(a, b):
        assert np.allclose(u, v, rtol=1e-10, atol=1e-12 * np.max(np.abs(v)))


def _bh_loss(c, mu, x, g, G, beta, normals=None, eps=None):
    T = oracle.Tree(c.points, c.normals if normals is None else normals, c.areas,
                    c.eps if eps is None else eps)
    T.update(mu)
    D, cnt = T.forward(x, beta, counters=True)
    return np.sum(g * D) + np.sum(G * T.forward_grad(x, beta)), cnt


def test_bh_geom_gradients_match_central_differences_of_bh_sum():
    """The far test uses p~ and r~ only, so perturbing n_m or eps_m keeps every
    decision (checked through the counters) and the Barnes-Hut sum is smooth in them."""
    w, c, x, g, G = _small_case(seed=2, n_q=80)
    beta = 1.5
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(w.mu)
    _, c0 = T.forward(x, beta, counters=True)
    assert c0[:, 1].sum() > 0  # some nodes are far
    dmu, dn, deps = T.adjoint_geom(x, beta, g, G)
    rng = np.random.default_rng(4)
    picks = list(rng.choice(c.n, 3, replace=False)) + list(np.argsort(-np.abs(deps))[:3])
    for m in picks:
        for k in range(3):
            nrm = c.normals.astype(np.float32).copy()
            vp, vm, st = _step(nrm[m, k], 1e-3)
            nrm[m, k] = vp
            lp, cp = _bh_loss(c, w.mu, x, g, G, beta, normals=nrm)
            nrm[m, k] = vm
            lm, cm = _bh_loss(c, w.mu, x, g, G, beta, normals=nrm)
            assert np.array_equal(cp, c0) and np.array_equal(cm, c0)
            assert abs((lp - lm) / st - dn[m, k]) <= 1e-7 * (1 + abs(dn[m, k]))
        e = c.eps.astype(np.float32).copy()
        vp, vm, st = _step(e[m], 1e-4 * e[m])
        e[m] = vp
        lp, _ = _bh_loss(c, w.mu, x, g, G, beta, eps=e)
        e[m] = vm
        lm, _ = _bh_loss(c, w.mu, x, g, G, beta, eps=e)
        # rounding of L itself limits the difference quotient to ~1e-13 |L| / step;
        # eps~ of a leaf is a float sum (the oracle's reading R7), whose rounding moves by whole
        # float units under a step of 1e-4 eps_m: 2e-4 relative
        assert abs((lp - lm) / st - deps[m]) <= 2e-4 * abs(deps[m]) + 1e-13 * abs(lp) / st


def test_linearity_in_normals_and_in_mu():
    """D and grad D are linear in the normals (point terms and n~) and in mu:
    sum_m n_m . dL/dn_m = sum_m mu_m . dL/dmu_m = <g, D> + <G, grad D>."""
    w = syn.workload("scene-200k", scale=0.02)
    c = w.cloud
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(w.mu)
    q = w.queries[:3000]
    rng = np.random.default_rng(5)
    g = rng.normal(size=(len(q), 4))
    G = rng.normal(size=(len(q), 4, 3))
    L = np.sum(g * T.forward(q, 2.0)) + np.sum(G * T.forward_grad(q, 2.0))
    dmu, dn, _ = T.adjoint_geom(q, 2.0, g, G)
    ln = np.sum(c.normals.astype(np.float32).astype(np.float64) * dn)
    lm = np.sum(w.mu.astype(np.float64) * dmu)
    assert abs(ln - L) <= 1e-10 * np.sum(np.abs(dn)) + 1e-12
    assert abs(lm - L) <= 1e-10 * np.sum(np.abs(dmu)) + 1e-12
    # the mu part is the existing adjoint of (D, grad D)
    assert np.allclose(dmu, T.adjoint_grad(q, 2.0, g, G), rtol=1e-12, atol=1e-14)


def _blurred_ball(s, R, eps):
    a, b = (R - s) / eps, (R + s) / eps
    return 0.5 * (math.erf(a) + math.erf(b)) - eps / (2 * s * math.sqrt(math.pi)) * (
        math.exp(-a * a) - math.exp(-b * b))


def test_global_eps_gradient_of_blurred_ball_closed_form():
    """Prop. 1: with one global eps, D on a dense sphere is the blurred ball
    indicator W(s; eps); the sum over points of dD/deps_m is dW/deps (central
    differences of the closed form)."""
    eps, R, n = 0.15, 1.0, 40000
    cl = syn.sphere_cloud(n, seed=0, eps=eps, radius=R, fibonacci=True)
    s_list = [0.3, 0.8, 0.95, 1.05, 1.3]
    dirs = syn._unit(np.random.default_rng(6).normal(size=(len(s_list), 3)))
    q = (np.array(s_list)[:, None] * dirs).astype(np.float32)
    for j, s in enumerate(np.linalg.norm(q.astype(np.float64), axis=1)):
        g = np.zeros((len(q), 1))
        g[j, 0] = 1.0
        _, _, deps = oracle.brute_adjoint_geom(cl.points, cl.normals, cl.areas, cl.eps,
                                               np.ones(n), q, g, None)
        h = 1e-5
        ref = (_blurred_ball(s, R, eps + h) - _blurred_ball(s, R, eps - h)) / (2 * h)
        assert abs(deps.sum() - ref) <= 5e-4, (s, deps.sum(), ref)


def test_eps_zero_has_zero_eps_gradient():
    w, c, x, g, G = _small_case(seed=7)
    _, dn, deps = oracle.brute_adjoint_geom(c.points, c.normals, c.areas, None, w.mu, x, g, G)
    assert np.all(deps == 0.0)
    assert np.any(dn != 0.0)
