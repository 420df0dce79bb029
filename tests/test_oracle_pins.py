"""Pins for the oracle: facts fixed by the paper and by mathematics, not by the
oracle's own formulas.  Each test names what it pins and where it comes from.

These run on the CPU only (no GPU) and are chosen so that a plausible slip in
the oracle (a dropped term of rho, a wrong sign, a missing 1/(4 pi), a wrong
epsilon convention, a transposed operand in the adjoint, a wrong ancestor set
in stage 2) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.special as sp

import oracle
from paper_2405_16788_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


# ---------------------------------------------------------------- rho ------

def test_rho_is_gaussian_ball_mass():
    """rho(t) equals the mass of the Gaussian exp(-r^2/eps^2)/(pi^1.5 eps^3) inside
    radius r = t eps, i.e. the regularized lower incomplete gamma P(3/2, t^2)
    (scipy).  Pins both terms of rho and their factors (Sec. 4.1)."""
    for t in np.concatenate([np.linspace(0.05, 6.0, 120), [0.3, 1.0, 2.5, 10.0]]):
        ref = sp.gammainc(1.5, t * t)
        assert abs(oracle.rho(t) - ref) < 1e-13 + 1e-11 * ref, t


def test_rho_derivative_identity():
    """rho'(t) = (4/sqrt(pi)) t^2 exp(-t^2) (central differences)."""
    for t in [0.2, 0.7, 1.3, 2.2, 3.1]:
        h = 1e-5
        fd = (oracle.rho(t + h) - oracle.rho(t - h)) / (2 * h)
        assert abs(fd - 4 / math.sqrt(math.pi) * t * t * math.exp(-t * t)) < 1e-8


def test_rho_limits_from_paper():
    """rho(0) = 0, rho(inf) = 1, and the finite value at the origin printed in
    Sec. 4.1: rho(r/eps) / (4 pi r^3) -> 3^-1 eps^-3 pi^-3/2 (golden fixture)."""
    g = _golden()
    assert oracle.rho(0.0) == 0.0
    assert oracle.rho(50.0) == g["rho_limits"]["rho_infinity"]
    t = 1e-2  # the next series term is -3t^2/5 relative
    val = oracle.rho(t) / (4 * math.pi * t ** 3)
    assert abs(val / g["rho_origin_limit"]["value_eps1"] - 1) < 2e-4


# ------------------------------------------------- single dipole, Prop. 2 ---

def _gaussian_smeared_dipole(x, p, n, eps, ns=96, nth=48, nph=96):
    """E[P(x, p + Z)], Z ~ N(0, eps^2/2 I), by quadrature in spherical
    coordinates centred at x, where the 1/s^2 of the kernel cancels the
    Jacobian: E = (1/4pi) int ds int dOmega (n . u) phi(x + s u - p)."""
    r = np.linalg.norm(np.asarray(x) - np.asarray(p))
    smax = r + 7 * eps
    sg, sw = np.polynomial.legendre.leggauss(ns)
    # split [0, smax] into 8 panels for accuracy
    edges = np.linspace(0, smax, 9)
    s = np.concatenate([(b - a) / 2 * sg + (a + b) / 2 for a, b in zip(edges[:-1], edges[1:])])
    w_s = np.concatenate([(b - a) / 2 * sw for a, b in zip(edges[:-1], edges[1:])])
    cg, cw = np.polynomial.legendre.leggauss(nth)
    ph = (np.arange(nph) + 0.5) * 2 * math.pi / nph
    ct = cg[:, None]
    st = np.sqrt(1 - ct * ct)
    u = np.stack([st * np.cos(ph)[None, :], st * np.sin(ph)[None, :],
                  np.broadcast_to(ct, (nth, nph))], axis=-1)  # [nth, nph, 3]
    w_ang = cw[:, None] * (2 * math.pi / nph)
    nu = u @ np.asarray(n)
    y = np.asarray(x)[None, None, None, :] + s[:, None, None, None] * u[None]
    d2 = np.sum((y - np.asarray(p)) ** 2, axis=-1)
    phi = np.exp(-d2 / eps ** 2) / (math.pi ** 1.5 * eps ** 3)
    return float(np.sum(w_s[:, None, None] * w_ang[None] * nu[None] * phi) / (4 * math.pi))


@pytest.mark.parametrize("t", [0.4, 1.0, 1.7, 3.0])
def test_single_dipole_matches_gaussian_noise_expectation(t):
    """Prop. 2 (Sec. 4.2): the expected singular kernel of a point whose position
    is Gaussian equals the regularized kernel.  With rho as printed, the noise
    has per-axis variance eps^2/2 (reading of the eps convention)."""
    eps = 0.3
    p = np.array([0.1, -0.2, 0.05])
    nrm = np.array([0.48, 0.6, 0.64])
    d = np.array([0.6, -0.3, 0.742])
    d /= np.linalg.norm(d)
    x = p + t * eps * d
    ref = _gaussian_smeared_dipole(x, p, nrm, eps)
    got = oracle.brute_forward(p[None], nrm[None], [1.0], [eps], [1.0], x[None].astype(np.float32))
    # the query is rounded to float32 on its way in; compare at that x
    xf = x.astype(np.float32).astype(np.float64)
    ref = _gaussian_smeared_dipole(xf, p.astype(np.float32).astype(np.float64),
                                   nrm.astype(np.float32).astype(np.float64), float(np.float32(eps)))
    assert abs(got[0, 0] - ref) < 2e-6 * max(abs(ref), 1e-3), (got, ref)


def test_single_dipole_singular_limit_is_solid_angle_density():
    """eps = 0: one dipole gives n.(p-x)/(4 pi |p-x|^3) (eq. pcwn); at x = p + r n
    this is -1/(4 pi r^2), the solid-angle density of a small patch seen head on."""
    for r in [0.1, 0.5, 2.0]:
        x = np.array([[0.0, 0.0, r]], np.float32)
        got = oracle.brute_forward([[0, 0, 0]], [[0, 0, 1]], [1.0], None, [1.0], x)[0, 0]
        rf = float(x[0, 2])
        assert abs(got + 1 / (4 * math.pi * rf * rf)) < 1e-12 / rf ** 2


# ------------------------------------------------------------ sphere -------

def _blurred_ball(s, R, eps):
    """Indicator of a ball of radius R blurred by the Gaussian of Prop. 1,
    evaluated at distance s from the centre (non-central chi, 3 d.o.f.)."""
    a = (R - s) / eps
    b = (R + s) / eps
    return 0.5 * (math.erf(a) + math.erf(b)) - eps / (2 * s * math.sqrt(math.pi)) * (
        math.exp(-a * a) - math.exp(-b * b))


def test_sphere_regularized_winding_number_is_blurred_indicator():
    """Prop. 1 (Sec. 4.1, App. A.1): the regularized winding number of a closed
    surface is its indicator blurred by a Gaussian.  A dense Fibonacci sphere
    (spacing 0.018 << eps = 0.15) reproduces the closed form at any distance,
    including on and near the surface."""
    eps, R, n = 0.15, 1.0, 40000
    cl = syn.sphere_cloud(n, seed=0, eps=eps, radius=R, fibonacci=True)
    s_list = [0.1, 0.5, 0.85, 0.95, 1.0, 1.05, 1.2, 1.6, 2.5]
    dirs = syn._unit(np.random.default_rng(5).normal(size=(len(s_list), 3)))
    q = (np.array(s_list)[:, None] * dirs).astype(np.float32)
    got = oracle.brute_forward(cl.points, cl.normals, cl.areas, cl.eps, np.ones(n), q)[:, 0]
    for s, gv in zip(s_list, got):
        ref = _blurred_ball(s, R, eps)
        assert abs(gv - ref) < 2e-4, (s, gv, ref)


def test_gauss_lemma_small_eps():
    """Eq. (gauss): about 1 inside and 0 outside, away from the surface."""
    g = _golden()["gauss_lemma"]
    cl = syn.sphere_cloud(40000, seed=0, eps=0.02, fibonacci=True)
    rng = np.random.default_rng(7)
    dirs = syn._unit(rng.normal(size=(40, 3)))
    rad = np.concatenate([rng.uniform(0.0, 0.75, 20), rng.uniform(1.25, 3.0, 20)])
    q = (rad[:, None] * dirs).astype(np.float32)
    got = oracle.brute_forward(cl.points, cl.normals, cl.areas, cl.eps, np.ones(cl.n), q)[:, 0]
    assert np.all(np.abs(got[:20] - g["inside"]) < 1e-3)
    assert np.all(np.abs(got[20:] - g["outside"]) < 1e-3)


def test_sign_flips_with_normals():
    """Inward normals negate the field (the kernel is linear in n)."""
    cl = syn.sphere_cloud(2000, seed=3, eps=0.05)
    q = syn.uniform_box_queries(64, seed=4)
    a = oracle.brute_forward(cl.points, cl.normals, cl.areas, cl.eps, np.ones(cl.n), q)
    b = oracle.brute_forward(cl.points, -cl.normals, cl.areas, cl.eps, np.ones(cl.n), q)
    assert np.allclose(a, -b, rtol=0, atol=1e-14)


# -------------------------------------------------------------- disk -------

def test_flat_disk_solid_angle():
    """A densely sampled disk (radius a, normal +z, eps = 0) seen from its axis at
    height h: D = -sign(h) (1/2)(1 - |h|/sqrt(h^2 + a^2)), the signed solid
    angle over 4 pi (eq. pcwn)."""
    a, nr, nt = 1.0, 300, 600
    r_mid = (np.arange(nr) + 0.5) * a / nr
    th = (np.arange(nt) + 0.5) * 2 * math.pi / nt
    R, TH = np.meshgrid(r_mid, th, indexing="ij")
    pts = np.stack([R * np.cos(TH), R * np.sin(TH), np.zeros_like(R)], -1).reshape(-1, 3)
    area = (R * (a / nr) * (2 * math.pi / nt)).reshape(-1)
    nrm = np.broadcast_to([0.0, 0.0, 1.0], pts.shape)
    hs = np.array([0.3, -0.3, 1.0, -2.0, 5.0])
    q = np.stack([np.zeros_like(hs), np.zeros_like(hs), hs], -1).astype(np.float32)
    got = oracle.brute_forward(pts, nrm, area, None, np.ones(len(area)), q)[:, 0]
    ref = -np.sign(hs) * 0.5 * (1 - np.abs(hs) / np.sqrt(hs ** 2 + a * a))
    assert np.allclose(got, ref, rtol=2e-5, atol=1e-6), (got, ref)


def test_eps_to_zero_gives_poisson_kernel():
    """Sec. 4.1: P_eps -> P as eps -> 0, pointwise away from the points."""
    cl = syn.sphere_cloud(3000, seed=9, eps=None)
    q = (syn._unit(np.random.default_rng(1).normal(size=(32, 3))) *
         np.random.default_rng(2).uniform(0.3, 0.8, (32, 1))).astype(np.float32)
    mu = syn.attributes(cl.n, 2, seed=3, kind="unit01")
    sing = oracle.brute_forward(cl.points, cl.normals, cl.areas, None, mu, q)
    for e in [1e-2, 1e-3]:
        reg = oracle.brute_forward(cl.points, cl.normals, cl.areas, np.full(cl.n, e), mu, q)
        # query-to-point distance >= 0.2: 1 - rho(0.2/eps) is below 1e-80
        assert np.allclose(reg, sing, rtol=0, atol=1e-12)


# ------------------------------------------------------ Barnes-Hut ---------

def _cfg1(scale=1.0):
    return syn.workload("sphere-2k", scale)


def test_bh_equals_brute_force_when_nothing_is_far():
    """Alg. 1 with beta -> infinity opens every node: BH is the exact sum."""
    w = _cfg1()
    c = w.cloud
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(w.mu)
    bh = T.forward(w.queries, np.inf)
    bf = oracle.brute_forward(c.points, c.normals, c.areas, c.eps, w.mu, w.queries)
    assert np.allclose(bh, bf, rtol=1e-12, atol=1e-14)


def test_bh_single_point_leaves_far_field_is_exact_per_point():
    """With single-point leaves (the paper's tree, Sec. 6.1) a leaf has radius 0,
    so it is always far and its far field (eq. farfield) is that point's exact
    term, up to the float rounding of the leaf's sums (the oracle's reading R7): a two-point
    cloud with leaf size 1, queried inside beta times the root radius,
    reproduces brute force."""
    p = np.array([[0.0, 0, 0], [0.3, 0.1, -0.2]], np.float32)
    n = np.array([[0, 0, 1.0], [0.6, 0.8, 0]], np.float32)
    a = np.array([0.2, 0.5], np.float32)
    e = np.array([0.05, 0.1], np.float32)
    mu = np.array([[1.5], [-0.7]], np.float32)
    T = oracle.Tree(p, n, a, e, leaf_size=1)
    T.update(mu)
    # queries near the pair: the root (r~ > 0) is opened, the two leaves (r~ = 0) are far
    q = np.array([[0.1, 0.0, 0.0], [0.2, 0.2, 0.1], [0.0, 0.05, 0.2]], np.float32)
    bh, cnt = T.forward(q, 2.0, counters=True)
    bf = oracle.brute_forward(p, n, a, e, mu, q)
    assert np.all(cnt[:, 1] == 2)
    assert np.allclose(bh, bf, rtol=1e-6, atol=1e-12)


def test_bh_error_shrinks_with_beta():
    """The far field is an approximation whose error falls as beta grows."""
    w = _cfg1()
    c = w.cloud
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(w.mu)
    bf = oracle.brute_forward(c.points, c.normals, c.areas, c.eps, w.mu, w.queries)
    errs = []
    for beta in [1.0, 2.0, 4.0, 8.0]:
        bh = T.forward(w.queries, beta)
        errs.append(np.max(np.abs(bh - bf)) / np.max(np.abs(bf)))
    assert errs[0] > errs[1] > errs[2] > errs[3], errs
    assert errs[3] < 1e-2


def test_bh_complexity_is_logarithmic():
    """Sec. 6.2: O(log M) per query.  Mean tested nodes grows far slower than N."""
    means = []
    for n in [2000, 16000, 128000]:
        cl = syn.sphere_cloud(n, seed=11, eps=0.02)
        T = oracle.Tree(cl.points, cl.normals, cl.areas, cl.eps)
        T.update(np.ones(n, np.float32))
        q = syn.uniform_box_queries(512, seed=12)
        _, cnt = T.forward(q, 2.0, counters=True)
        means.append(cnt[:, 0].mean() + cnt[:, 2].mean())
    assert means[2] / means[0] < 6.0, means  # linear would be 64x


def test_bh_adjoint_is_transpose_of_forward():
    """<g, K mu> = <K^T g, mu> for BH at beta = 2: the two-stage adjoint (Sec.
    5.2, eqs. farfield_gradient and farfield_features_gradient) is the exact
    transpose of the Barnes-Hut forward map, which is linear in mu."""
    w = syn.workload("scene-200k", scale=0.02)
    c = w.cloud
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(w.mu)
    q = w.queries[:3000]
    y = T.forward(q, 2.0)
    g = syn.upstream_grad(len(q), w.mu.shape[1], seed=5).astype(np.float64)
    gm = T.adjoint(q, 2.0, g)
    lhs = float(np.sum(g * y))
    rhs = float(np.sum(gm * w.mu.astype(np.float64)))
    assert abs(lhs - rhs) < 1e-11 * (abs(lhs) + np.sum(np.abs(g * y))), (lhs, rhs)


def test_bh_adjoint_matches_finite_differences():
    """Central differences of the BH forward map in mu_m (exact for a linear
    map up to rounding) on a few points."""
    w = syn.workload("sphere-2k", scale=0.25)
    c = w.cloud
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    mu = w.mu.astype(np.float64)
    T.update(mu.astype(np.float32))
    g = syn.upstream_grad(len(w.queries), 1, seed=8).astype(np.float64)
    gm = T.adjoint(w.queries, 2.0, g)
    rng = np.random.default_rng(0)
    for m in rng.choice(c.n, 6, replace=False):
        h = 0.25
        mp, mm = mu.copy(), mu.copy()
        mp[m, 0] += h
        mm[m, 0] -= h
        mp32, mm32 = mp.astype(np.float32), mm.astype(np.float32)
        T.update(mp32)
        yp = T.forward(w.queries, 2.0)
        T.update(mm32)
        ym = T.forward(w.queries, 2.0)
        # the step actually taken after rounding the attributes to float32
        step = float(mp32[m, 0]) - float(mm32[m, 0])
        fd = np.sum(g * (yp - ym)) / step
        assert abs(fd - gm[m, 0]) < 1e-9 * (1 + abs(fd)), (m, fd, gm[m, 0])


def test_bh_adjoint_equals_brute_adjoint_when_nothing_is_far():
    w = syn.workload("sphere-2k", scale=0.5)
    c = w.cloud
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(w.mu)
    g = syn.upstream_grad(len(w.queries), 1, seed=9)
    a = T.adjoint(w.queries, np.inf, g)
    b = oracle.brute_adjoint(c.points, c.normals, c.areas, c.eps, w.queries, g)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-14)


def test_brute_adjoint_matches_finite_differences():
    w = syn.workload("sphere-2k", scale=0.1)
    c = w.cloud
    g = syn.upstream_grad(len(w.queries), 2, seed=10).astype(np.float64)
    mu = syn.attributes(c.n, 2, seed=11, kind="unit01").astype(np.float64)
    ga = oracle.brute_adjoint(c.points, c.normals, c.areas, c.eps, w.queries, g)
    for m in [0, 17, 150]:
        for ch in [0, 1]:
            mp, mm = mu.copy(), mu.copy()
            mp[m, ch] += 0.5
            mm[m, ch] -= 0.5
            yp = oracle.brute_forward(c.points, c.normals, c.areas, c.eps, mp, w.queries)
            ym = oracle.brute_forward(c.points, c.normals, c.areas, c.eps, mm, w.queries)
            step = float(np.float32(mp[m, ch])) - float(np.float32(mm[m, ch]))
            fd = np.sum(g * (yp - ym)) / step
            assert abs(fd - ga[m, ch]) < 1e-9 * (1 + abs(fd))


def test_node_moments_follow_definition():
    """Eqs. (farfield_dipole), (farfield_dipole_features) at the root: A~ = sum A,
    p~ = sum A p / A~, r~ = max |p - p~|, and the far field of the root seen from
    far away tends to the brute-force sum (the cluster acts as one dipole)."""
    w = syn.workload("scene-200k", scale=0.01)
    c = w.cloud
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(w.mu)
    e = T.export()
    A = c.areas.astype(np.float64)
    P = c.points.astype(np.float64)
    # leaves sum in float (the oracle's reading R7): a few float roundings of the exact sums
    assert abs(e["area"][0] - A.sum()) < 1e-6 * A.sum()
    cen = (A[:, None] * P).sum(0) / A.sum()
    assert np.allclose(e["cen"][0], cen, rtol=0, atol=2e-6)
    rmax = np.max(np.linalg.norm(P - e["cen32"][0].astype(np.float64), axis=1))
    assert abs(e["r32"][0] - rmax) <= 2e-7 * rmax
    far = (np.array([[40.0, -25.0, 31.0]]) * np.array([[1.0], [3.0], [9.0]])).astype(np.float32)
    bh = T.forward(far, 2.0)
    bf = oracle.brute_forward(c.points, c.normals, c.areas, c.eps, w.mu, far)
    rel = np.abs(bh - bf) / np.abs(bf)
    assert np.all(rel[0] < 0.05) and np.all(rel[2] < rel[0] + 1e-9)


def test_far_test_is_strict_and_scales_with_beta():
    """Alg. 1's far test ||x - p~|| > beta r~ (reading: strict).  Values chosen
    so that every float operation is exact: a 3-4-5 triangle."""
    c = [0.0, 0.0, 0.0]
    assert not oracle.far_test([3.0, 4.0, 0.0], c, 2.5, 2.0)   # on the sphere: not far
    assert oracle.far_test([3.0, 4.0, 0.125], c, 2.5, 2.0)     # just outside
    assert not oracle.far_test([3.0, 3.875, 0.0], c, 2.5, 2.0)  # just inside
    assert oracle.far_test([3.0, 4.0, 0.0], c, 2.5, 1.5)       # beta scales the radius
    assert not oracle.far_test([3.0, 4.0, 0.0], c, 2.5, 2.5)
    assert oracle.far_test([0.0, 0.0, 1e-3], c, 0.0, 2.0)      # a zero-radius node is far ...
    assert not oracle.far_test(c, c, 0.0, 2.0)                 # ... unless the query is on it
    # the offset is taken from the node centre, per axis
    assert not oracle.far_test([10.0, 20.0, 30.0], [7.0, 16.0, 30.0], 2.5, 2.0)
    assert oracle.far_test([10.0, 20.0, 30.0], [7.0, 16.0, 29.5], 2.5, 2.0)


def test_near_tie_diagnostic_counts_boundary_queries():
    """The oracle reports far tests within 1e-6 d of the boundary |x - p~| = beta r~
    (reading R6's diagnostic): a query placed on a node's boundary sphere is
    counted there; one placed at twice that distance is not counted at that node."""
    p = np.array([[0.0, 0.0, 0.0], [0.6, 0.2, -0.1]], np.float32)
    n = np.array([[0, 0, 1], [1, 0, 0]], np.float32)
    A = np.array([0.3, 0.7], np.float32)
    T = oracle.Tree(p, n, A, None, leaf_size=1)
    T.update(np.ones((2, 1), np.float32))
    ex = T.export()
    c, r = ex["cen32"][0].astype(np.float64), float(ex["r32"][0])
    u = np.array([0.36, 0.48, 0.8])
    on = (c + 2.0 * r * (1 + 1e-9) * u).astype(np.float32)[None]
    off = (c + 4.0 * r * u).astype(np.float32)[None]
    assert T.near_ties(on, 2.0)[0] >= 1
    assert T.near_ties(off, 2.0)[0] == 0
