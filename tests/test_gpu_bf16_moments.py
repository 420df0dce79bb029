"""bf16 node moments (DIPOLE_BF16_MOMENTS) on every form of the value forward
that reads them: the dense grid (its bricks walk the same kernel) and the
planned forward agree with the plain forward on the same tree; switching a
tree between storages reallocates its attribute state and gives each
storage's own results; the gradient forward keeps the float moments."""
import numpy as np
import pytest

from paper_2405_16788_gb300 import synthetic as syn
from _helpers import bf16_round, gpu_tree, normwise, oracle_tree, to_dev
from test_gpu_grid import _grid_points

pytestmark = pytest.mark.gpu


def test_grid_and_planned_forward_read_the_bf16_moments():
    import torch
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("scene-200k", scale=0.05)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu).to(torch.bfloat16), bf16_moments=True)
    dims, lo = (33, 21, 17), (-1.2, -1.1, -1.0)
    h = 2.3 / max(dims)
    yg = gt.forward_grid(lo, h, dims, 2.0).cpu().numpy().reshape(-1, 4)
    pts = _grid_points(lo, h, dims)
    X = to_dev(pts)
    y = gt.forward(X, 2.0).cpu().numpy()
    plan = dipole.QueryPlan(len(pts), X.device)
    yp = gt.forward(X, 2.0, plan=plan).cpu().numpy()
    gt.sync_status()
    assert np.all(normwise(yg, y) <= 1e-6), normwise(yg, y)
    assert np.all(normwise(yp, y) <= 1e-6), normwise(yp, y)
    # and they are the bf16-moment results, not the float-moment ones
    ot = oracle_tree(w.cloud)
    ot.update(bf16_round(w.mu), bf16_moments=True)
    ref_m, allow = ot.forward_bf16_allowance(pts, 2.0)
    assert np.all(np.max(np.abs(y - ref_m) - allow, axis=0) / np.max(np.abs(ref_m), axis=0) <= 1e-4)


def test_switching_storage_reallocates_and_changes_the_results():
    import torch
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("scene-200k", scale=0.05)
    gt = gpu_tree(w.cloud)
    X = to_dev(w.queries[:8000])
    mu_b = to_dev(w.mu).to(torch.bfloat16)
    outs = {}
    for kind in ("m16", "bf16", "f32", "m16"):
        if kind == "f32":
            gt.refit(to_dev(w.mu))
        else:
            gt.refit(mu_b, bf16_moments=kind == "m16")
        info = dipole.dipole_tree_info_get(gt.handle)
        want = {"m16": dipole.DIPOLE_BF16_MOMENTS, "bf16": dipole.DIPOLE_BF16, "f32": dipole.DIPOLE_F32}
        assert info["dtype"] == want[kind]
        y = gt.forward(X, 2.0).cpu().numpy()
        if kind in outs:
            assert np.array_equal(y, outs[kind])  # the same storage gives the same bits again
        outs[kind] = y
    gt.sync_status()
    assert not np.array_equal(outs["m16"], outs["bf16"])
    ot = oracle_tree(w.cloud)
    ot.update(bf16_round(w.mu))
    ref_b = ot.forward(w.queries[:8000], 2.0)
    assert np.all(normwise(outs["bf16"], ref_b) <= 1e-4)


def test_gradient_forward_keeps_the_float_moments():
    import torch
    w = syn.workload("scene-200k", scale=0.05)
    q = w.queries[:6000]
    X = to_dev(q)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(w.mu).to(torch.bfloat16), bf16_moments=True)
    d16, g16 = gt.forward_grad(X, 2.0)
    gt.refit(to_dev(w.mu).to(torch.bfloat16))
    d, g = gt.forward_grad(X, 2.0)
    gt.sync_status()
    assert np.array_equal(g16.cpu().numpy(), g.cpu().numpy())
    assert np.array_equal(d16.cpu().numpy(), d.cpu().numpy())
