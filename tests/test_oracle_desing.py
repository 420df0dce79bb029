"""Pins for the oracle's desingularized kernel (the oracle's reading R11: 1/r^3 ->
1/max(r, eps)^3, the paper's ablation baseline): equality with the singular
kernel outside every cutoff, the closed form inside one, Barnes-Hut = brute
force when nothing is far, and its gradients against central differences."""
import math

import numpy as np

import oracle
from paper_2405_16788_gb300 import synthetic as syn


def test_outside_every_cutoff_equals_the_singular_kernel():
    w = syn.workload("scene-200k", scale=0.01)
    c = w.cloud
    q = np.array([[1.9, 0.1, 0.2], [-1.7, 1.2, 0.0], [0.0, 0.0, 1.99]], np.float32)
    with oracle.kernel("desingularized"):
        d = oracle.brute_forward(c.points, c.normals, c.areas, c.eps, w.mu, q)
    s = oracle.brute_forward(c.points, c.normals, c.areas, None, w.mu, q)
    assert np.array_equal(d, s)


def test_inside_the_cutoff_closed_form():
    eps, A, mu = 0.2, 0.7, 1.3
    n = np.array([[0.0, 0.6, 0.8]])
    x = np.array([[0.03, -0.05, 0.02]], np.float32)
    with oracle.kernel("desingularized"):
        d = oracle.brute_forward([[0.0, 0, 0]], n, [A], [eps], [mu], x)[0, 0]
        g = oracle.brute_forward_grad([[0.0, 0, 0]], n, [A], [eps], [mu], x)[0, 0]
    u = -x[0].astype(np.float64)
    f = lambda v: float(np.float32(v))  # the oracle takes float inputs
    A32, e32, mu32 = f(A), f(eps), f(mu)
    n32 = n[0].astype(np.float32).astype(np.float64)
    assert math.isclose(d, A32 * mu32 * float(n32 @ u) / (4 * math.pi * e32 ** 3), rel_tol=1e-12)
    # inside the cutoff the kernel is linear in x: gradient -A mu n / (4 pi eps^3)
    assert np.allclose(g, -A32 * mu32 * n32 / (4 * math.pi * e32 ** 3), rtol=1e-12)
    # and it differs from the regularized kernel there
    d_reg = oracle.brute_forward([[0.0, 0, 0]], n, [A], [eps], [mu], x)[0, 0]
    assert abs(d_reg - d) > 1e-3 * abs(d)


def test_bh_equals_brute_when_nothing_is_far():
    w = syn.workload("sphere-2k", scale=0.5)
    c = w.cloud
    with oracle.kernel("desingularized"):
        T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
        T.update(w.mu)
        a = T.forward(w.queries, np.inf)
        b = oracle.brute_forward(c.points, c.normals, c.areas, c.eps, w.mu, w.queries)
        ga = T.forward_grad(w.queries, np.inf)
        gb = oracle.brute_forward_grad(c.points, c.normals, c.areas, c.eps, w.mu, w.queries)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-13)
    assert np.allclose(ga, gb, rtol=1e-11, atol=1e-13)


def test_gradients_match_central_differences():
    """grad_x against differences of D (queries kept off the cutoff spheres);
    d/deps_m and d/dn_m against differences of L = <g, D> + <G, grad D>."""
    w = syn.workload("scene-200k", scale=0.004)
    c = w.cloud
    rng = np.random.default_rng(0)
    near = c.points[rng.choice(c.n, 30)] + rng.normal(scale=0.006, size=(30, 3))
    x = np.concatenate([near, rng.uniform(-1.2, 1.2, size=(30, 3))]).astype(np.float32)
    with oracle.kernel("desingularized"):
        g = oracle.brute_forward_grad(c.points, c.normals, c.areas, c.eps, w.mu, x)
        h = 1e-6
        for k in range(3):
            xp, xm = x.astype(np.float64).copy(), x.astype(np.float64).copy()
            xp[:, k] += h
            xm[:, k] -= h
            xp32, xm32 = xp.astype(np.float32), xm.astype(np.float32)
            dp = oracle.brute_forward(c.points, c.normals, c.areas, c.eps, w.mu, xp32)
            dm = oracle.brute_forward(c.points, c.normals, c.areas, c.eps, w.mu, xm32)
            st = (xp32[:, k].astype(np.float64) - xm32[:, k].astype(np.float64))[:, None]
            fd = (dp - dm) / st
            scale = np.max(np.abs(g[:, :, k]), axis=0)
            assert np.all(np.max(np.abs(fd - g[:, :, k]), axis=0) <= 1e-4 * scale)
        gu = rng.normal(size=(len(x), 4))
        G = rng.normal(size=(len(x), 4, 3))
        _, dn, deps = oracle.brute_adjoint_geom(c.points, c.normals, c.areas, c.eps, w.mu, x, gu, G)

        def L(nrm=c.normals, e=c.eps):
            D = oracle.brute_forward(c.points, nrm, c.areas, e, w.mu, x)
            GD = oracle.brute_forward_grad(c.points, nrm, c.areas, e, w.mu, x)
            return np.sum(gu * D) + np.sum(G * GD)

        for m in np.argsort(-np.abs(deps))[:4]:
            e = c.eps.astype(np.float32).copy()
            ep, em = np.float32(e[m] * (1 + 1e-4)), np.float32(e[m] * (1 - 1e-4))
            e[m] = ep
            lp = L(e=e)
            e[m] = em
            lm = L(e=e)
            fd = (lp - lm) / (float(ep) - float(em))
            assert abs(fd - deps[m]) <= 1e-5 * abs(deps[m]), (m, fd, deps[m])
            nrm = c.normals.astype(np.float32).copy()
            vp, vm = np.float32(nrm[m, 0] + 1e-3), np.float32(nrm[m, 0] - 1e-3)
            nrm[m, 0] = vp
            lp = L(nrm=nrm)
            nrm[m, 0] = vm
            lm = L(nrm=nrm)
            assert abs((lp - lm) / (float(vp) - float(vm)) - dn[m, 0]) <= 1e-7 * (1 + abs(dn[m, 0]))
