"""The rendering loop around the dipole sums (camera rays with the exact
attenuation of eq. surface_density, free-flight entropy, shadow rays to a point
light): the gradient of the loss with respect to the attributes, through the
library's forward and adjoint of D and grad D, against central differences of
the same loss evaluated in double from the oracle's Barnes-Hut; and a short
Adam loop that reduces the loss, in float32 and in bfloat16 attributes."""
import math

import numpy as np
import pytest
from scipy.special import log_ndtr

import oracle
from paper_2405_16788_gb300 import synthetic as syn
from _helpers import normwise, oracle_tree, to_dev

pytestmark = pytest.mark.gpu
S_SCALE = 10.0
LAMBDA_H = 1e-3


def _np_sigma(D0, gD0, om, s):
    z = s * (0.5 - D0)
    ratio = np.exp(-0.5 * z * z - 0.5 * math.log(2 * math.pi) - log_ndtr(z))
    return s * ratio * np.abs(np.sum(om * gD0, axis=-1))


def _np_ff(sigma, delta):
    tau = sigma * delta
    acc = np.cumsum(tau, axis=-1)
    p = np.exp(-(acc - tau)) * (-np.expm1(-tau))
    return p, np.exp(-acc[..., -1])


def _np_shadow(xs, light, jit, offset=0.05, clip=1.5):
    K = jit.shape[1]
    to_l = light[None, :] - xs
    dist = np.linalg.norm(to_l, axis=1)
    w = to_l / dist[:, None]
    b = np.sum(xs * w, axis=1)
    c = np.sum(xs * xs, axis=1) - clip * clip
    t_end = np.maximum(np.minimum(dist, -b + np.sqrt(np.maximum(b * b - c, 0))), offset + 1e-4)
    ts = offset + (np.arange(K)[None, :] + jit) * ((t_end - offset)[:, None] / K)
    d = np.diff(ts, axis=1, prepend=np.full((len(xs), 1), offset))
    return xs[:, None, :] + ts[..., None] * w[:, None, :], w, d


class _OracleScene:
    """The loss in double: D and grad D from the oracle's Barnes-Hut."""

    def __init__(self, w, scale_rays):
        o, d, t = w.meta["rays"]
        self.o, self.d, self.t = o, d, t
        self.R, self.S = t.shape
        self.delta = np.diff(t, axis=1, prepend=w.meta["t_near"][:, None])
        self.X = w.queries
        self.light = w.meta["light"]
        self.jit = w.meta["shadow_jitter"]
        self.tree = oracle_tree(w.cloud)

    def fields(self, mu, idx=None):
        R, S = self.R, self.S
        self.tree.update(mu)
        D = self.tree.forward(self.X, 2.0).reshape(R, S, -1)
        G = self.tree.forward_grad(self.X, 2.0).reshape(R, S, -1, 3)
        sig = _np_sigma(D[..., 0], G[..., 0, :], self.d[:, None, :], S_SCALE)
        p, _ = _np_ff(sig, self.delta)
        if idx is None:
            idx = np.argmax(p, axis=1)
        xs = self.X.reshape(R, S, 3)[np.arange(R), idx].astype(np.float64)
        Xs, wsh, dsh = _np_shadow(xs, self.light, self.jit)
        Xs32 = Xs.reshape(-1, 3).astype(np.float32)
        Ds = self.tree.forward(Xs32, 2.0).reshape(R, -1, D.shape[-1])
        Gs = self.tree.forward_grad(Xs32, 2.0).reshape(R, -1, D.shape[-1], 3)
        return D, G, Ds, Gs, idx, xs, Xs32, wsh, dsh

    def loss_from(self, D, G, Ds, Gs, idx, xs, wsh, dsh, target):
        R = self.R
        ar = np.arange(R)
        sig = _np_sigma(D[..., 0], G[..., 0, :], self.d[:, None, :], S_SCALE)
        p, _ = _np_ff(sig, self.delta)
        col = np.sum(p[..., None] * D[..., 1:4], axis=1)
        H = -np.sum(p * np.log(np.maximum(p, 1e-12)), axis=1)
        sig_sh = _np_sigma(Ds[..., 0], Gs[..., 0, :], wsh[:, None, :], S_SCALE)
        _, T_sh = _np_ff(sig_sh, dsh)
        gf = -G[ar, idx, 0, :]
        n_hat = gf / np.maximum(np.linalg.norm(gf, axis=1, keepdims=True), 1e-12)
        to_l = self.light[None, :] - xs
        dist = np.linalg.norm(to_l, axis=1)
        cosine = np.maximum(np.sum(n_hat * to_l, axis=1) / dist, 0.0)
        direct = D[ar, idx, 1:4] * (T_sh * cosine / dist ** 2)[:, None]
        col = col + p.sum(1)[:, None] * direct
        if target is None:
            return col
        return np.mean(np.abs(col - target)) + LAMBDA_H * np.mean(H)


def _renderer(w, **kw):
    import torch
    from paper_2405_16788_gb300 import render
    o, d, t = w.meta["rays"]
    c = w.cloud
    f = lambda a: to_dev(np.asarray(a, np.float32))
    return render.Renderer(f(c.points), f(c.normals), f(c.areas), f(c.eps), f(o), f(d), f(t),
                           f(w.meta["t_near"]), f(w.meta["light"]), n_shadow=64,
                           shadow_jitter=f(w.meta["shadow_jitter"]), s=S_SCALE,
                           queries=to_dev(w.queries), **kw)


def test_render_loss_gradient_matches_oracle_finite_differences():
    import torch
    w = syn.workload("scene-5m-loop", scale=0.002)  # 10,000 points, 16 rays x 192, 64 shadow
    mu_gt = w.mu
    mu = (mu_gt + np.random.default_rng(9).normal(scale=0.05, size=mu_gt.shape)).astype(np.float32)
    sc = _OracleScene(w, 1.0)
    f = sc.fields(mu_gt)
    target = sc.loss_from(*f[:6], f[7], f[8], None)
    D, G, Ds, Gs, idx, xs, Xs32, wsh, dsh = sc.fields(mu)
    L0 = sc.loss_from(D, G, Ds, Gs, idx, xs, wsh, dsh, target)

    rd = _renderer(w)
    attrs = to_dev(mu).requires_grad_(True)
    L, _ = rd.loss(attrs, to_dev(target.astype(np.float32)), LAMBDA_H,
                   shadow_index=torch.from_numpy(idx).cuda())
    assert abs(float(L.detach()) - L0) <= 1e-3 * abs(L0), (float(L.detach()), L0)
    L.backward()
    grad = attrs.grad.cpu().numpy().astype(np.float64)

    # columns of the linear maps mu -> D, grad D for 64 sampled points (one-hot attributes)
    pts = np.random.default_rng(10).choice(w.cloud.n, 64, replace=False)
    onehot = np.zeros((w.cloud.n, 64), np.float32)
    onehot[pts, np.arange(64)] = 1.0
    sc.tree.update(onehot)
    K = sc.tree.forward(sc.X, 2.0).reshape(sc.R, sc.S, 64)
    KG = sc.tree.forward_grad(sc.X, 2.0).reshape(sc.R, sc.S, 64, 3)
    Ks = sc.tree.forward(Xs32, 2.0).reshape(sc.R, -1, 64)
    KGs = sc.tree.forward_grad(Xs32, 2.0).reshape(sc.R, -1, 64, 3)
    h = 1e-4
    fd = np.zeros((64, 4))
    for j in range(64):
        for ch in range(4):
            args = []
            for sgn in (1.0, -1.0):
                Dp, Gp, Dsp, Gsp = D.copy(), G.copy(), Ds.copy(), Gs.copy()
                Dp[..., ch] += sgn * h * K[..., j]
                Gp[..., ch, :] += sgn * h * KG[..., j, :]
                Dsp[..., ch] += sgn * h * Ks[..., j]
                Gsp[..., ch, :] += sgn * h * KGs[..., j, :]
                args.append(sc.loss_from(Dp, Gp, Dsp, Gsp, idx, xs, wsh, dsh, target))
            fd[j, ch] = (args[0] - args[1]) / (2 * h)
    err = normwise(grad[pts], fd)
    assert np.all(err <= 1e-3), err  # the gradient tolerance (measured ~5e-6)


@pytest.mark.parametrize("dtype", ["float32", "bfloat16"])
def test_adam_loop_reduces_the_loss(dtype):
    import torch
    from paper_2405_16788_gb300 import render
    w = syn.workload("scene-5m-loop", scale=0.01)  # 50,000 points, 82 rays
    rd = _renderer(w)
    with torch.no_grad():
        target, _, _ = rd.render(to_dev(w.mu))
    mu0 = w.mu.copy()
    mu0[:, 0] = 1.0  # geometry attributes start at 1 (the regularized winding number)
    mu0[:, 1:] = np.random.default_rng(3).normal(scale=0.3, size=(w.cloud.n, 3)) + 0.5
    _, losses = render.train(rd, to_dev(mu0.astype(np.float32)), target, steps=40, lr=2e-2,
                             attr_dtype=getattr(torch, dtype))
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.7 * losses[0], losses
    rd.tree.sync_status()
