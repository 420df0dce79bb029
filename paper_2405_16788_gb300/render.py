"""Differentiable volume rendering around the dipole sums: the inverse-rendering
loop that the fast queries serve (Sec. 3 and Sec. 5 of arXiv 2405.16788).

Everything here is PyTorch elementwise work on the outputs of the library's
queries; the dipole sums and their gradients run in libdipole through
``dipole.dipole_sum_and_grad``.  The pieces, in the paper's notation:

* geometry field ``f = 1/2 - D^0`` (eq. geometry_field) from the first channel;
* vacancy ``v = Phi(s f)`` (eq. vacancy) and attenuation
  ``sigma = |omega . grad v| / v`` (eq. surface_density), with
  ``grad v = -phi(s f) s grad D^0``: the exact spatial gradient of the dipole sum;
* quadrature (eq. quadrature) in the standard form of the exponential volume
  rendering equation (eq. rendering): ``T_j = exp(-sum_{i<j} sigma_i Delta_i)``,
  ``p_j = T_j (1 - exp(-sigma_j Delta_j))``; the printed form has a sign typo in
  the second factor and lets the first sum run to j;
* free-flight entropy ``H = -sum_j p_j log p_j`` (App. entropy, eq. shannon_entropy);
* one shadow ray per camera ray, from the sample of largest ``p_j`` to a point
  light, with direct light ``albedo T(x, l) n^.(l - x)/|l - x|^3`` (eq. direct),
  ``n^ = grad f/|grad f|`` the implicit normal and ``T`` the transmittance by the
  same quadrature.
* radiance: the appearance channels ``D^1..3`` themselves stand in for the
  paper's MLP (eq. radiance_field), which is not part of the fast summation.
"""
from __future__ import annotations

import math

import torch

from . import dipole

_LOG_SQRT_2PI = 0.5 * math.log(2.0 * math.pi)


def vacancy_sigma(D0: torch.Tensor, gD0: torch.Tensor, dirs: torch.Tensor, s: float):
    """v = Phi(s (1/2 - D0)) and sigma = |dirs . grad v| / v.

    D0 [...], gD0 [..., 3] (grad of D^0), dirs broadcastable to gD0.  phi/Phi is
    taken as exp(log phi - log Phi), which stays finite deep inside (s f << 0)."""
    z = s * (0.5 - D0)
    v = torch.special.ndtr(z)
    ratio = torch.exp(-0.5 * z * z - _LOG_SQRT_2PI - torch.special.log_ndtr(z))  # phi(z)/Phi(z)
    sigma = s * ratio * (dirs * gD0).sum(-1).abs()
    return v, sigma


def free_flight(sigma: torch.Tensor, delta: torch.Tensor):
    """p_j = T_j (1 - exp(-sigma_j delta_j)) and the transmittance past the last
    sample, along the last axis."""
    tau = sigma * delta
    acc = torch.cumsum(tau, dim=-1)
    T = torch.exp(-(acc - tau))  # exp(-sum_{i<j} tau_i)
    p = T * (-torch.expm1(-tau))
    return p, torch.exp(-acc[..., -1])


def entropy(p: torch.Tensor, tiny: float = 1e-12):
    """Shannon entropy of each ray's free-flight weights (eq. shannon_entropy)."""
    return -(p * torch.log(p.clamp_min(tiny))).sum(-1)


def sample_deltas(t: torch.Tensor, t_near: torch.Tensor):
    """Delta_j = t_j - t_{j-1} with t_0 = t_near."""
    return torch.diff(t, dim=-1, prepend=t_near[..., None])


def shadow_samples(xs: torch.Tensor, light: torch.Tensor, jitter: torch.Tensor,
                   offset: float = 0.05, clip_radius: float = 1.5):
    """K = jitter.shape[1] stratified samples on each segment from xs + offset
    toward the light, ending at the light or where the segment leaves the clip
    sphere: (queries [R, K, 3], unit directions [R, 3], deltas [R, K])."""
    K = jitter.shape[1]
    to_l = light.reshape(1, 3) - xs
    dist = to_l.norm(dim=-1)
    w = to_l / dist[:, None]
    b = (xs * w).sum(-1)
    c = (xs * xs).sum(-1) - clip_radius ** 2
    t_exit = -b + torch.sqrt(torch.clamp(b * b - c, min=0.0))
    t_end = torch.minimum(dist, t_exit).clamp_min(offset + 1e-4)
    j = torch.arange(K, device=xs.device, dtype=xs.dtype)[None, :]
    ts = offset + (j + jitter) * ((t_end - offset)[:, None] / K)
    X = xs[:, None, :] + ts[..., None] * w[:, None, :]
    return X, w, sample_deltas(ts, torch.full_like(t_end, offset))


def direct_light(albedo, T, grad_D0, xs, light):
    """eq. direct: albedo T n^.(l - x)/|l - x|^3 with n^ = grad f/|grad f|,
    grad f = -grad D^0, clamped at 0 for points facing away from the light."""
    gf = -grad_D0
    n_hat = gf / gf.norm(dim=-1, keepdim=True).clamp_min(1e-12)
    to_l = light.reshape(1, 3) - xs
    dist = to_l.norm(dim=-1)
    cosine = ((n_hat * to_l).sum(-1) / dist).clamp_min(0.0)
    return albedo * (T * cosine / (dist * dist))[:, None]


class Renderer:
    """Renders rays through a dipole-sum scene and differentiates the result
    with respect to the per-point attributes (geometry channel 0, RGB 1..3).

    The tree is built once from the fixed positions, normals, areas and radii
    (the paper trains attributes with the geometry held fixed between point
    growing stages) and refit from the attributes on every render."""

    def __init__(self, points, normals, areas, radii, origins, dirs, t, t_near, light,
                 n_shadow: int = 64, shadow_jitter=None, s: float = 10.0, beta: float = 2.0,
                 shadow_offset: float = 0.05, clip_radius: float = 1.5, leaf_size: int = 8,
                 queries=None):
        self.tree = dipole.DipoleTree(points, normals, areas, radii, leaf_size=leaf_size)
        self.o, self.d, self.t, self.t_near = origins, dirs, t, t_near
        self.R, self.S = t.shape
        if queries is None:  # the ray samples o + t d, ray-major
            queries = (origins[:, None, :] + t[..., None] * dirs[:, None, :]).reshape(-1, 3)
        self.X = queries.reshape(-1, 3).contiguous()
        self.delta = sample_deltas(t, t_near)
        self.light = light.reshape(3)
        self.K = int(n_shadow)
        if shadow_jitter is None:
            shadow_jitter = torch.full((self.R, self.K), 0.5, device=t.device)
        self.jit = shadow_jitter
        self.s, self.beta = float(s), float(beta)
        self.offset, self.clip = float(shadow_offset), float(clip_radius)

    def render(self, attrs: torch.Tensor, shadow_index: torch.Tensor | None = None):
        """Pixel colours [R, 3], per-ray entropy [R] and the shadow-ray origin
        index [R] (the sample of largest p_j unless given)."""
        R, S = self.R, self.S
        D, G = dipole.dipole_sum_and_grad(attrs, self.tree, self.X, self.beta)
        D, G = D.reshape(R, S, -1), G.reshape(R, S, -1, 3)
        _, sigma = vacancy_sigma(D[..., 0], G[..., 0, :], self.d[:, None, :], self.s)
        p, _ = free_flight(sigma, self.delta)
        colour = (p[..., None] * D[..., 1:4]).sum(1)
        H = entropy(p)
        if shadow_index is None:
            shadow_index = torch.argmax(p.detach(), dim=1)
        ar = torch.arange(R, device=p.device)
        xs = self.X.reshape(R, S, 3)[ar, shadow_index]
        Xs, w, dsh = shadow_samples(xs, self.light, self.jit, self.offset, self.clip)
        Ds, Gs = dipole.dipole_sum_and_grad(attrs, self.tree, Xs.reshape(-1, 3).contiguous(),
                                            self.beta, refit=False)
        _, sig_sh = vacancy_sigma(Ds.reshape(R, self.K, -1)[..., 0],
                                  Gs.reshape(R, self.K, -1, 3)[..., 0, :], w[:, None, :], self.s)
        _, T_sh = free_flight(sig_sh, dsh)
        direct = direct_light(D[ar, shadow_index, 1:4], T_sh, G[ar, shadow_index, 0, :], xs,
                              self.light)
        colour = colour + p.sum(1)[:, None] * direct
        return colour, H, shadow_index

    def loss(self, attrs, target, entropy_weight: float = 1e-3, shadow_index=None):
        colour, H, idx = self.render(attrs, shadow_index)
        return (colour - target).abs().mean() + entropy_weight * H.mean(), idx


def train(renderer: Renderer, attrs0: torch.Tensor, target: torch.Tensor, steps: int,
          lr: float = 1e-2, entropy_weight: float = 1e-3, attr_dtype=torch.float32,
          callback=None):
    """Adam on the per-point attributes (float32 master copy; the kernels read
    them in attr_dtype, e.g. bfloat16).  Returns the attributes and the losses."""
    master = attrs0.detach().to(torch.float32).clone().requires_grad_(True)
    opt = torch.optim.Adam([master], lr=lr)
    losses = []
    for it in range(steps):
        opt.zero_grad(set_to_none=True)
        L, _ = renderer.loss(master.to(attr_dtype), target, entropy_weight)
        L.backward()
        opt.step()
        losses.append(float(L.detach()))
        if callback is not None:
            callback(it, losses[-1])
    return master.detach(), losses
