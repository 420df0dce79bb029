"""Shared helpers for the GPU parity tests: move synthetic inputs to the GPU,
build the GPU tree and the oracle tree from the same arrays, and the
norm-wise error metric used by every tolerance."""
from __future__ import annotations

import numpy as np

import oracle


def to_dev(a, dev="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def gpu_tree(cloud, leaf_size=8, max_depth=10):
    from paper_2405_16788_gb300 import dipole
    return dipole.DipoleTree(to_dev(cloud.points), to_dev(cloud.normals), to_dev(cloud.areas),
                             None if cloud.eps is None else to_dev(cloud.eps),
                             leaf_size=leaf_size, max_depth=max_depth)


def oracle_tree(cloud, leaf_size=8, max_depth=10):
    return oracle.Tree(cloud.points, cloud.normals, cloud.areas, cloud.eps, leaf_size=leaf_size,
                       max_depth=max_depth)


def normwise(y, ref):
    """Per channel: max_q |y - ref| / max_q |ref| (the parity metric)."""
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    if y.ndim == 1:
        y, ref = y[:, None], ref[:, None]
    den = np.max(np.abs(ref), axis=0)
    den = np.where(den > 0, den, 1.0)
    return np.max(np.abs(y - ref), axis=0) / den


def excess_over_allowance(y, ref, allow):
    """Per channel: the largest max_q (|y - ref| - allow) / max_q |ref|, the
    norm-wise error once each element may differ by its allowance (the bf16
    roundings that both implementations may take either way)."""
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.max(np.abs(ref), axis=0)
    den = np.where(den > 0, den, 1.0)
    return np.max(np.abs(y - ref) - allow, axis=0) / den


def bf16_round(a):
    """Round float32 to bfloat16 (nearest even) and back, in numpy."""
    a = np.ascontiguousarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)
