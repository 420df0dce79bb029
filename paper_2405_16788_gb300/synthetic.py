"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs: point clouds with normals, area weights and
regularization radii, per-point attributes, ray-sample query points and
upstream gradients.  It holds none of the dipole-sum arithmetic, so both the
CUDA path and the CPU oracle take their inputs from here.

The paper's scenes are dense structure-from-motion point clouds of the DTU and
BlendedMVS datasets (Sec. 7), which are not available; the procedural clouds
below stand in for them: a noisy torus and two spheres, outliers uniform in a
box, jittered normals, and (for the largest workload) anisotropic density.
Area weights are the component area divided by its point count (the paper
estimates them as in Barill et al. 2018, which it does not restate); outliers
take the median inlier weight.  Queries are stratified samples along camera
rays (Sec. 7.1, "ray sampling").

All generators use ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _unit(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def uniform_sphere(rng, n: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """n points uniform by area on a sphere, and their outward unit normals."""
    nrm = _unit(rng.normal(size=(n, 3)))
    return np.asarray(center) + radius * nrm, nrm


def fibonacci_sphere(n: int, radius: float = 1.0):
    """Deterministic, nearly even sphere sampling (golden-angle spiral)."""
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    phi = math.pi * (1.0 + math.sqrt(5.0)) * i
    rxy = np.sqrt(1.0 - z * z)
    nrm = np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1)
    return radius * nrm, nrm


def uniform_torus(rng, n: int, R: float, r: float):
    """n points uniform by area on a torus around the z axis (rejection sampling)."""
    out_p, out_n, have = [], [], 0
    while have < n:
        k = 2 * (n - have) + 64
        th = rng.uniform(0, 2 * math.pi, k)
        ph = rng.uniform(0, 2 * math.pi, k)
        keep = rng.uniform(0, 1, k) < (R + r * np.cos(ph)) / (R + r)
        th, ph = th[keep], ph[keep]
        nrm = np.stack([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph)], axis=1)
        ctr = np.stack([R * np.cos(th), R * np.sin(th), np.zeros_like(th)], axis=1)
        out_p.append(ctr + r * nrm)
        out_n.append(nrm)
        have += len(th)
    return np.concatenate(out_p)[:n], np.concatenate(out_n)[:n]


@dataclass
class Cloud:
    """An oriented point cloud with area weights and regularization radii (float32)."""
    points: np.ndarray
    normals: np.ndarray
    areas: np.ndarray
    eps: np.ndarray | None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.points.shape[0])


def sphere_cloud(n: int, seed: int, eps: float | None = 0.02, radius: float = 1.0,
                 fibonacci: bool = False) -> Cloud:
    """A sampled sphere with exact outward normals and equal area weights."""
    if fibonacci:
        p, nrm = fibonacci_sphere(n, radius)
    else:
        p, nrm = uniform_sphere(_rng(seed), n, radius)
    a = np.full(n, 4 * math.pi * radius * radius / n)
    e = None if eps is None else np.full(n, eps)
    return Cloud(p.astype(np.float32), nrm.astype(np.float32), a.astype(np.float32),
                 None if e is None else e.astype(np.float32), dict(kind="sphere"))


def scene_cloud(n: int, seed: int, outlier_frac: float = 0.05, noise: float = 0.005,
                eps_range=(0.002, 0.02), anisotropic: bool = False) -> Cloud:
    """Noisy union of a torus (R=0.6, r=0.2, z=0 plane) and two spheres (radius 0.3
    at (0, 0, +-0.55)) plus outliers uniform in [-1,1]^3; normals jittered by
    N(0, 0.1^2) and renormalized; radii log-uniform in eps_range.

    anisotropic=True: the torus is sampled 10x denser (per unit area) than the
    spheres and density falls along z as exp(-2z) (rejection), the shape of a
    dense SfM cloud whose coverage varies across the scene.
    """
    rng = _rng(seed)
    n_out = int(round(outlier_frac * n))
    n_in = n - n_out
    comps = [("torus", 4 * math.pi ** 2 * 0.6 * 0.2), ("sphere+", 4 * math.pi * 0.09),
             ("sphere-", 4 * math.pi * 0.09)]
    dens = np.array([10.0, 1.0, 1.0]) if anisotropic else np.ones(3)
    share = np.array([a for _, a in comps]) * dens
    counts = np.floor(share / share.sum() * n_in).astype(int)
    counts[0] += n_in - counts.sum()
    ps, ns, As = [], [], []
    for (name, area), k in zip(comps, counts):
        if anisotropic:  # oversample, then keep with probability exp(-2 (z - zmax))
            pool_p, pool_n, have = [], [], 0
            while have < k:
                m = 3 * (k - have) + 64
                if name == "torus":
                    p, nr = uniform_torus(rng, m, 0.6, 0.2)
                else:
                    c = (0, 0, 0.55) if name == "sphere+" else (0, 0, -0.55)
                    p, nr = uniform_sphere(rng, m, 0.3, c)
                keep = rng.uniform(0, 1, m) < np.exp(-2.0 * (p[:, 2] - 0.85))
                pool_p.append(p[keep])
                pool_n.append(nr[keep])
                have += int(keep.sum())
            p, nr = np.concatenate(pool_p)[:k], np.concatenate(pool_n)[:k]
        elif name == "torus":
            p, nr = uniform_torus(rng, k, 0.6, 0.2)
        else:
            c = (0, 0, 0.55) if name == "sphere+" else (0, 0, -0.55)
            p, nr = uniform_sphere(rng, k, 0.3, c)
        ps.append(p)
        ns.append(nr)
        As.append(np.full(k, area / max(k, 1)))
    p = np.concatenate(ps)
    nrm = np.concatenate(ns)
    A = np.concatenate(As)
    p = p + rng.normal(scale=noise, size=p.shape)
    nrm = _unit(nrm + rng.normal(scale=0.1, size=nrm.shape))
    if n_out:
        po = rng.uniform(-1, 1, size=(n_out, 3))
        no = _unit(rng.normal(size=(n_out, 3)))
        ao = np.full(n_out, np.median(A))
        p = np.concatenate([p, po])
        nrm = np.concatenate([nrm, no])
        A = np.concatenate([A, ao])
    lo, hi = eps_range
    e = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))
    perm = rng.permutation(n)  # input order carries no spatial structure
    return Cloud(p[perm].astype(np.float32), nrm[perm].astype(np.float32),
                 A[perm].astype(np.float32), e.astype(np.float32),
                 dict(kind="scene", outliers=n_out, anisotropic=anisotropic))


def camera_rays(n_rays: int, seed: int, cam_radius: float = 2.5, fov_deg: float = 50.0,
                clip_radius: float = 1.5, origin=None):
    """Random cameras on a sphere looking at the origin, random pixels: returns
    (origins [R,3], unit directions [R,3], t_near [R], t_far [R]) with every
    ray clipped to the sphere of radius clip_radius."""
    rng = _rng(seed)
    cam = _unit(rng.normal(size=(n_rays, 3))) * cam_radius
    if origin is not None:
        cam = np.broadcast_to(np.asarray(origin, np.float64), (n_rays, 3)).copy()
    fwd = _unit(-cam)
    helper = np.where(np.abs(fwd[:, 2:3]) < 0.9, np.array([[0, 0, 1.0]]), np.array([[1.0, 0, 0]]))
    right = _unit(np.cross(fwd, helper))
    up = np.cross(right, fwd)
    tan_h = math.tan(math.radians(fov_deg) / 2)
    u = rng.uniform(-1, 1, size=(n_rays, 1)) * tan_h
    v = rng.uniform(-1, 1, size=(n_rays, 1)) * tan_h
    d = _unit(fwd + u * right + v * up)
    b = np.sum(cam * d, axis=1)
    c = np.sum(cam * cam, axis=1) - clip_radius ** 2
    disc = np.maximum(b * b - c, 0.0)
    t_n = np.maximum(-b - np.sqrt(disc), 0.0)
    t_f = -b + np.sqrt(disc)
    return cam, d, t_n, t_f


def stratified_samples(origins, dirs, t_n, t_f, n_samples: int, seed: int):
    """t_j = t_n + (j + u_j)(t_f - t_n)/S along each ray: queries [R*S, 3] float32
    (ray-major, samples contiguous along each ray) and t [R, S]."""
    rng = _rng(seed)
    R = origins.shape[0]
    j = np.arange(n_samples)[None, :]
    u = rng.uniform(0, 1, size=(R, n_samples))
    t = t_n[:, None] + (j + u) * ((t_f - t_n)[:, None] / n_samples)
    x = origins[:, None, :] + t[..., None] * dirs[:, None, :]
    return x.reshape(-1, 3).astype(np.float32), t


def uniform_box_queries(q: int, seed: int, half: float = 1.5) -> np.ndarray:
    return _rng(seed).uniform(-half, half, size=(q, 3)).astype(np.float32)


def attributes(n: int, C: int, seed: int, kind: str = "scene") -> np.ndarray:
    """Per-point attributes [n, C] float32.  kind='unit01': U(0,1) in every
    channel.  kind='scene': channel 0 geometry ~ U(0.5, 1.5), channels 1-3 RGB
    ~ U(0,1), further feature channels ~ N(0,1)."""
    rng = _rng(seed)
    if kind == "unit01":
        return rng.uniform(0, 1, size=(n, C)).astype(np.float32)
    out = np.empty((n, C), np.float32)
    out[:, 0] = rng.uniform(0.5, 1.5, n)
    k = min(C, 4)
    if k > 1:
        out[:, 1:k] = rng.uniform(0, 1, size=(n, k - 1))
    if C > 4:
        out[:, 4:] = rng.normal(size=(n, C - 4))
    return out


def upstream_grad(q: int, C: int, seed: int) -> np.ndarray:
    """A seeded stand-in for dL/dD [q, C] float32 (N(0,1))."""
    return _rng(seed).normal(size=(q, C)).astype(np.float32)


@dataclass
class Workload:
    name: str
    cloud: Cloud
    mu: np.ndarray
    queries: np.ndarray
    beta: float = 2.0
    leaf_size: int = 8
    attr_dtype: str = "f32"
    meta: dict = field(default_factory=dict)


WORKLOADS = {
    "sphere-2k": "N=2,000 points uniform on the unit sphere, eps=0.02, C=1 U(0,1); "
                 "Q=4,096 uniform in [-1.5,1.5]^3; beta=2, leaf size 8",
    "scene-200k": "N=200,000 noisy torus+2 spheres, 5% outliers, eps log-U[0.002,0.02], C=4; "
                  "Q=8,192 rays x 128 stratified samples",
    "scene-1m": "N=1,000,000 noisy torus+2 spheres, 2% outliers, eps log-U[0.002,0.02], C=4 f32; "
                "Q=4,096 rays x 128 stratified samples = 524,288; beta=2, leaf 8",
    "scene-3m-bf16": "N=3,000,000, 3% outliers, C=16 (1+3+12) stored bf16; Q=16,384 rays x 128",
    "scene-5m-loop": "N=5,000,000 anisotropic density, 5% outliers, C=4; per step 8,192 camera "
                     "rays x 192 + 8,192 shadow rays x 64 to a point light at (1.8, 1.2, 2.2)",
}


def workload(name: str, scale: float = 1.0) -> Workload:
    """The named workload.  scale < 1 shrinks N and the ray count (for quick runs)."""
    def sz(k):
        return max(1, int(round(k * scale)))

    if name == "sphere-2k":
        cl = sphere_cloud(sz(2000), seed=1001, eps=0.02)
        mu = attributes(cl.n, 1, seed=2001, kind="unit01")
        qs = uniform_box_queries(sz(4096), seed=3001)
        return Workload(name, cl, mu, qs)
    if name == "scene-200k":
        cl = scene_cloud(sz(200_000), seed=1002, outlier_frac=0.05)
        mu = attributes(cl.n, 4, seed=2002)
        o, d, tn, tf = camera_rays(sz(8192), seed=3002)
        qs, _ = stratified_samples(o, d, tn, tf, 128, seed=4002)
        return Workload(name, cl, mu, qs)
    if name == "scene-1m":
        cl = scene_cloud(sz(1_000_000), seed=1003, outlier_frac=0.02)
        mu = attributes(cl.n, 4, seed=2003)
        o, d, tn, tf = camera_rays(sz(4096), seed=3003)
        qs, t = stratified_samples(o, d, tn, tf, 128, seed=4003)
        return Workload(name, cl, mu, qs, meta=dict(rays=(o, d, t)))
    if name == "scene-3m-bf16":
        cl = scene_cloud(sz(3_000_000), seed=1004, outlier_frac=0.03)
        mu = attributes(cl.n, 16, seed=2004)
        o, d, tn, tf = camera_rays(sz(16384), seed=3004)
        qs, _ = stratified_samples(o, d, tn, tf, 128, seed=4004)
        return Workload(name, cl, mu, qs, attr_dtype="bf16")
    if name == "scene-5m-loop":
        cl = scene_cloud(sz(5_000_000), seed=1005, outlier_frac=0.05, anisotropic=True)
        mu = attributes(cl.n, 4, seed=2005)
        o, d, tn, tf = camera_rays(sz(8192), seed=3005)
        qs, t = stratified_samples(o, d, tn, tf, 192, seed=4005)
        # one point light outside the scene and the jitter of 64 stratified
        # samples on each shadow ray
        jit = _rng(5005).uniform(0, 1, size=(o.shape[0], 64))
        return Workload(name, cl, mu, qs, meta=dict(rays=(o, d, t), t_near=tn, t_far=tf,
                                                    light=np.array([1.8, 1.2, 2.2]),
                                                    shadow_jitter=jit))
    raise KeyError(name)
