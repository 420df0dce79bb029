"""Dense-grid primal queries (the evaluation grid that the paper meshes with
marching cubes, Sec. 7): the kernel generates the grid points itself; results
equal dipole_forward on the same points up to the rounding of the partial
sums (which are folded every 32 steps of the warp, so they depend on a query's
warp neighbours), with the same traversal, and the oracle within 1e-4."""
import numpy as np
import pytest

from paper_2405_16788_gb300 import synthetic as syn
from _helpers import gpu_tree, normwise, oracle_tree, to_dev

pytestmark = pytest.mark.gpu


def _grid_points(lo, h, dims):
    """lo + ((float)i * h) per axis in float32, one rounding per operation."""
    lo = np.asarray(lo, np.float32)
    h = np.float32(h)
    ax = [lo[d] + np.arange(dims[d]).astype(np.float32) * h for d in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.stack([x, y, z], -1).reshape(-1, 3).astype(np.float32)


@pytest.mark.parametrize("dims", [(37, 29, 23), (4, 4, 2), (1, 1, 1), (9, 1, 3), (64, 64, 64)])
def test_grid_equals_listed_queries_and_oracle(dims):
    w = syn.workload("scene-200k", scale=0.05)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    lo, h = (-1.2, -1.1, -1.0), 2.3 / max(dims)
    y = gt.forward_grid(lo, h, dims, 2.0).cpu().numpy()
    assert y.shape == (dims[2], dims[1], dims[0], 4)
    pts = _grid_points(lo, h, dims)
    ref_gpu = gt.forward(to_dev(pts), 2.0).cpu().numpy()
    assert np.all(normwise(y.reshape(-1, 4), ref_gpu) <= 1e-6), normwise(y.reshape(-1, 4), ref_gpu)
    ot = oracle_tree(w.cloud)
    ot.update(w.mu)
    sel = np.arange(len(pts)) if len(pts) <= 20000 else np.random.default_rng(0).choice(len(pts), 20000, replace=False)
    ref = ot.forward(pts[sel], 2.0)
    assert np.all(normwise(y.reshape(-1, 4)[sel], ref) <= 1e-4)
    gt.sync_status()


def test_grid_argument_errors():
    import torch
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("sphere-2k")
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    out = torch.empty(8, device="cuda")
    for lo, h, dims in [((0, 0, 0), 0.0, (2, 2, 2)), ((0, 0, 0), 0.1, (0, 2, 2)),
                        ((0, 0, float("nan")), 0.1, (2, 2, 2)), ((0, 0, 0), 0.1, (1 << 25, 1, 1))]:
        with pytest.raises(dipole.DipoleError):
            dipole.dipole_forward_grid(gt.handle, lo, h, dims, 2.0, out)


@pytest.mark.slow
def test_grid_512_full_size_sampled():
    """512^3 grid over the benchmark scene (1M points): 4096 sampled points
    against the oracle."""
    w = syn.workload("scene-1m")
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu))
    dims = (512, 512, 512)
    lo, h = (-1.5, -1.5, -1.5), np.float32(3.0 / 511)
    y = gt.forward_grid(lo, float(h), dims, 2.0)
    gt.sync_status()
    rng = np.random.default_rng(5)
    ijk = rng.integers(0, 512, size=(4096, 3))
    lo32 = np.asarray(lo, np.float32)
    pts = (lo32[None, :] + ijk.astype(np.float32) * h).astype(np.float32)
    got = y[ijk[:, 2], ijk[:, 1], ijk[:, 0]].cpu().numpy()
    ot = oracle_tree(w.cloud)
    ot.update(w.mu)
    assert np.all(normwise(got, ot.forward(pts, 2.0)) <= 1e-4)
