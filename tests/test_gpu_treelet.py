"""The treelet option (dipole_set_treelet): the value forward stages the upper
tree in shared memory.  It reads the same values from there as from global
memory and takes the same decisions, so every result is bit-identical with the
option off: plain, planned (ranged) and grid forwards, float and bf16
attributes, channels without the foreshortening term, and after a refit
(the staged moments follow).  Trees it does not cover (more than 4 channels)
run the plain kernels."""
import numpy as np
import pytest

from paper_2405_16788_gb300 import synthetic as syn
from _helpers import gpu_tree, to_dev
from test_gpu_grid import _grid_points

pytestmark = pytest.mark.gpu


def _forwards(gt, X, lo, h, dims):
    from paper_2405_16788_gb300 import dipole
    plan = dipole.QueryPlan(X.shape[0], X.device)
    out = [gt.forward(X, 2.0).cpu().numpy(), gt.forward(X, 2.0, plan=plan).cpu().numpy(),
           gt.forward_grid(lo, h, dims, 2.0).cpu().numpy()]
    gt.sync_status()
    return out


@pytest.mark.parametrize("C,G,bf16", [(4, 4, False), (1, 1, False), (3, 3, True), (4, 1, False), (8, 8, False)])
def test_treelet_results_are_bit_identical(C, G, bf16):
    import torch
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("scene-200k", scale=0.05)
    gt = gpu_tree(w.cloud)
    X = to_dev(w.queries[:20000])
    lo, h, dims = (-1.2, -1.1, -1.0), 0.05, (40, 31, 23)
    for seed in (C, C + 100):  # a refit between: the staged moments follow
        mu = to_dev(syn.attributes(w.cloud.n, C, seed=seed))
        if bf16:
            mu = mu.to(torch.bfloat16)
        gt.refit(mu, geometry_channels=None if G == C else G)
        dipole.dipole_set_treelet(gt.handle, False)
        off = _forwards(gt, X, lo, h, dims)
        dipole.dipole_set_treelet(gt.handle, True)
        on = _forwards(gt, X, lo, h, dims)
        for a, b in zip(off, on):
            assert np.array_equal(a, b)


def test_treelet_argument_errors():
    from paper_2405_16788_gb300 import dipole
    w = syn.workload("sphere-2k")
    gt = gpu_tree(w.cloud)
    with pytest.raises(dipole.DipoleError):
        dipole.dipole_set_treelet(0, True)
    lib = dipole.load_library()
    assert lib.dipole_set_treelet(__import__("ctypes").c_void_p(gt.handle), 2) == dipole.DIPOLE_EINVAL
