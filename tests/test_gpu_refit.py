"""GPU tree update (eq. farfield_dipole_features): the node moments
S_t^c = sum_{m in t} A_m n_m mu_m^c exported by the library, checked against
that definition summed in float64 over each node's points, plus the
refit's edge cases (channels of very different magnitude, an all-zero
channel, a tree that is a single leaf, a non-finite attribute, bf16 storage,
repeatability)."""
import numpy as np
import pytest

from paper_2405_16788_gb300 import dipole
from paper_2405_16788_gb300 import synthetic as syn
from _helpers import bf16_round, gpu_tree, normwise, oracle_tree, to_dev

pytestmark = pytest.mark.gpu


def _definition(cloud, mu, ex):
    """S and sum |A n mu| per node and column, float64, from the exported
    Morton permutation and point ranges."""
    perm = ex["perm"].astype(np.int64)
    w = (cloud.areas.astype(np.float64)[:, None] * cloud.normals.astype(np.float64))[perm]
    m = np.asarray(mu, np.float64)[perm]
    terms = (m[:, :, None] * w[:, None, :]).reshape(len(perm), -1)  # [N, 3C], column 3c + k
    S = np.zeros((len(ex["first"]), terms.shape[1]))
    B = np.zeros_like(S)
    for t, (f, k) in enumerate(zip(ex["first"], ex["count"])):
        S[t] = terms[f:f + k].sum(0)
        B[t] = np.abs(terms[f:f + k]).sum(0)
    return S, B


def _moments(gt):
    return dipole.dipole_tree_export(gt.handle, moments=True)


def _close(got, S, B, ex, cols=slice(None)):
    """A leaf sums its k points in float (error below k 2^-24 of sum |terms|);
    an internal node is the exact sum of its leaves' sums, rounded once."""
    k = np.where(ex["is_leaf"] == 1, np.maximum(ex["count"], 8), 8).astype(np.float64)[:, None]
    tol = k * 2.0 ** -22 * B[:, cols] + 1e-38
    return np.all(np.abs(np.asarray(got, np.float64)[:, cols] - S[:, cols]) <= tol)


def test_moments_follow_definition_across_scales():
    w = syn.workload("scene-200k", scale=0.1)
    mu = syn.attributes(w.cloud.n, 5, seed=3).astype(np.float64)
    mu *= np.array([1e6, 1.0, 1e-6, 1e-20, 0.0])  # the last channel is all zeros
    mu = mu.astype(np.float32)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(mu))
    ex = _moments(gt)
    S, B = _definition(w.cloud, mu, ex)
    got = ex["moments"].astype(np.float64)
    assert _close(got, S, B, ex), np.max(np.abs(got - S) / (B + 1e-300))
    assert np.all(got[:, 12:15] == 0.0)
    # and the queries see them: forward against the oracle, every channel
    ot = oracle_tree(w.cloud)
    ot.update(mu)
    q = w.queries[:4000]
    y = gt.forward(to_dev(q), 2.0).cpu().numpy()
    ref = ot.forward(q, 2.0)
    err = normwise(y[:, :4], ref[:, :4])
    assert np.all(err <= 1e-4), err
    assert np.all(y[:, 4] == 0.0)


def test_single_leaf_tree():
    rng = np.random.default_rng(7)
    cloud = syn.sphere_cloud(5, seed=7)
    mu = rng.normal(size=(5, 3)).astype(np.float32)
    gt = gpu_tree(cloud)
    gt.refit(to_dev(mu))
    ex = _moments(gt)
    assert len(ex["first"]) == 1 and ex["is_leaf"][0] == 1
    S, B = _definition(cloud, mu, ex)
    assert _close(ex["moments"], S, B, ex)
    q = rng.uniform(-1.5, 1.5, size=(300, 3)).astype(np.float32)
    ot = oracle_tree(cloud)
    ot.update(mu)
    assert np.all(normwise(gt.forward(to_dev(q), 2.0).cpu().numpy(), ot.forward(q, 2.0)) <= 1e-4)


def test_nonfinite_attribute_poisons_only_its_channel():
    w = syn.workload("sphere-2k")
    mu = syn.attributes(w.cloud.n, 3, seed=5)
    mu[17, 1] = np.nan
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(mu))
    ex = _moments(gt)
    got = ex["moments"]
    inner = ex["is_leaf"] == 0
    assert np.all(np.isnan(got[inner][:, 3:6]))
    clean = mu.copy()
    clean[:, 1] = 0.0
    S, B = _definition(w.cloud, clean, ex)
    keep = [0, 1, 2, 6, 7, 8]
    assert _close(got, S, B, ex, keep)


def test_bf16_attributes_moments():
    import torch
    w = syn.workload("scene-200k", scale=0.05)
    mu = syn.attributes(w.cloud.n, 4, seed=9)
    gt = gpu_tree(w.cloud)
    gt.refit(to_dev(mu).to(torch.bfloat16))
    ex = _moments(gt)
    S, B = _definition(w.cloud, bf16_round(mu), ex)
    assert _close(ex["moments"], S, B, ex)


def test_refit_is_repeatable_and_follows_new_attributes():
    w = syn.workload("scene-200k", scale=0.05)
    gt = gpu_tree(w.cloud)
    mu1 = syn.attributes(w.cloud.n, 4, seed=1)
    mu2 = syn.attributes(w.cloud.n, 4, seed=2)
    gt.refit(to_dev(mu1))
    a = _moments(gt)["moments"]
    gt.refit(to_dev(mu2))
    gt.refit(to_dev(mu1))
    b = _moments(gt)["moments"]
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    gt.refit(to_dev(mu2))
    ex = _moments(gt)
    S, B = _definition(w.cloud, mu2, ex)
    assert _close(ex["moments"], S, B, ex)
