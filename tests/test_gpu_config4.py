"""Mixed precision at full size: 3,000,000 points, 16 channels stored in
bfloat16, 2,097,152 queries.  On a 10,000-query subsample: the bf16 path
against the oracle on the bf16-rounded attributes (1e-4, the kernel's own
error), against the oracle on the float32 attributes (3e-3, max norm per
channel, wherever the bf16 rounding of the inputs alone stays within it; see
test_gpu_forward._bf16_gate), the float32 path on the same GPU (1e-4); the
adjoint (upstream gradient on the subsample only) 1e-3.  The same with bf16
node moments (DIPOLE_BF16_MOMENTS) against the oracle's reading R13, where an
element may differ in addition by the oracle's allowance for node sums on the
edge of a bf16 rounding boundary."""
import numpy as np
import pytest

from paper_2405_16788_gb300 import synthetic as syn
from _helpers import bf16_round, excess_over_allowance, gpu_tree, normwise, oracle_tree, to_dev
from test_gpu_forward import _bf16_gate

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_config4_bf16_full_size_subsample():
    import torch
    w = syn.workload("scene-3m-bf16")
    Q, C = len(w.queries), w.mu.shape[1]
    assert (w.cloud.n, Q, C) == (3_000_000, 2_097_152, 16)
    idx = np.random.default_rng(4).choice(Q, 10000, replace=False)
    gt = gpu_tree(w.cloud)
    X = to_dev(w.queries)
    gt.refit(to_dev(w.mu).to(torch.bfloat16))
    yb = gt.forward(X, 2.0)[torch.from_numpy(idx).cuda()].cpu().numpy()
    g = np.zeros((Q, C), np.float32)
    g[idx] = syn.upstream_grad(10000, C, seed=21)
    ga = gt.adjoint(X, 2.0, to_dev(g)).cpu().numpy()
    gt.refit(to_dev(w.mu))
    yf = gt.forward(X, 2.0)[torch.from_numpy(idx).cuda()].cpu().numpy()
    gt.sync_status()

    ot = oracle_tree(w.cloud)
    ot.update(bf16_round(w.mu))
    ref_b = ot.forward(w.queries[idx], 2.0)
    aref = ot.adjoint(w.queries[idx], 2.0, g[idx].astype(np.float64))
    ot.update(w.mu)
    ref_f = ot.forward(w.queries[idx], 2.0)
    assert np.all(normwise(yb, ref_b) <= 1e-4), normwise(yb, ref_b)
    assert np.all(normwise(yf, ref_f) <= 1e-4), normwise(yf, ref_f)
    assert np.all(normwise(ga, aref) <= 1e-3), normwise(ga, aref)
    _bf16_gate(normwise(yb, ref_f), normwise(ref_b, ref_f))


def test_config4_bf16_moments_full_size_subsample():
    import torch
    w = syn.workload("scene-3m-bf16")
    Q = len(w.queries)
    idx = np.random.default_rng(5).choice(Q, 10000, replace=False)
    gt = gpu_tree(w.cloud)
    X = to_dev(w.queries)
    gt.refit(to_dev(w.mu).to(torch.bfloat16), bf16_moments=True)
    ym = gt.forward(X, 2.0)[torch.from_numpy(idx).cuda()].cpu().numpy()
    gt.sync_status()
    ot = oracle_tree(w.cloud)
    ot.update(bf16_round(w.mu), bf16_moments=True)
    ref_m, allow = ot.forward_bf16_allowance(w.queries[idx], 2.0)
    ot.update(w.mu)
    ref_f = ot.forward(w.queries[idx], 2.0)
    ex = excess_over_allowance(ym, ref_m, allow)
    assert np.all(ex <= 1e-4), (ex, normwise(ym, ref_m), np.mean(allow > 0))
    _bf16_gate(normwise(ym, ref_f), normwise(ref_m, ref_f))
