"""Pins for the oracle's bf16 node moments (reading R13): the rounding against
PyTorch's own float -> bfloat16 conversion (a library routine, round to
nearest even), and the far field of a single far node against the definition
of the node sum (eq. farfield_dipole_features) rounded by that library routine."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_16788_gb300 import synthetic as syn

torch = pytest.importorskip("torch")


def _torch_bf16(x32):
    return torch.from_numpy(np.ascontiguousarray(x32, np.float32)).to(torch.bfloat16).to(
        torch.float64).numpy()


def test_round_bf16_matches_library_conversion():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-60, 60, 20000))).astype(np.float32)
    # exact ties, one below and one above, with even and odd kept parts
    hi = rng.integers(0, 1 << 16, 4000, dtype=np.uint64) << np.uint64(16)
    hi &= np.uint64(0x7F7F0000)  # finite exponents
    low = np.array([0x8000, 0x7FFF, 0x8001, 0x0000, 0xFFFF], np.uint64)
    u = (hi[:, None] | low[None, :]).ravel().astype(np.uint32)
    ties = u.view(np.float32)
    special = np.array([0.0, -0.0, 1.0, -1.0, 3.3895314e38, -3.3895314e38, np.finfo(np.float32).max,
                        np.finfo(np.float32).tiny, 1e-40, -1e-45, np.inf, -np.inf], np.float32)
    for v in (x, ties, -ties, special):
        got = oracle.round_bf16(v.astype(np.float64))
        np.testing.assert_array_equal(got, _torch_bf16(v))


def test_round_bf16_rounds_to_float_first():
    """R13 rounds to float, then to bf16.  1 + 2^-8 + 2^-30 rounds to the float
    1 + 2^-8, an exact tie between the bf16 values 1 and 1 + 2^-7, which goes to
    the even one (1); a single rounding of the double would give 1 + 2^-7."""
    x = np.array([1.0 + 2.0 ** -8 + 2.0 ** -30, -(1.0 + 2.0 ** -8 + 2.0 ** -30)])
    np.testing.assert_array_equal(oracle.round_bf16(x), [1.0, -1.0])
    x = np.array([1.0 + 3 * 2.0 ** -8])  # a tie above an odd kept part rounds up
    np.testing.assert_array_equal(oracle.round_bf16(x), [1.0 + 2.0 ** -6])


@pytest.mark.parametrize("G", [4, 1])
def test_root_far_field_uses_the_rounded_node_sums(G):
    """A query so far away that only the root is taken as far: with bf16 moments
    the oracle's D^c is (p~ - x) . round(S^c) / (4 pi d^3) for channels with
    the foreshortening term and round(sum A mu) / (4 pi d^2) without it (R12),
    S^c = sum_m A_m n_m mu_m^c summed here in float64 and rounded by PyTorch."""
    w = syn.workload("scene-200k", scale=0.01)
    c = w.cloud
    C = 4
    mu = syn.attributes(c.n, C, seed=3)
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    T.update(mu, geometry_channels=G, bf16_moments=True)
    e = T.export()
    x = np.array([[300.0, -170.0, 240.0]], np.float32)
    y, cnt = T.forward(x, 2.0, counters=True)
    assert cnt[0, 0] == 1 and cnt[0, 1] == 1  # the root alone, taken as far
    A = c.areas.astype(np.float64)
    N = c.normals.astype(np.float64)
    M = mu.astype(np.float64)
    S = np.einsum("m,mk,mc->ck", A, N, M)  # [C, 3]
    Sm = (A[:, None] * M).sum(0)            # [C]
    u = e["cen"][0] - x[0].astype(np.float64)
    d = np.linalg.norm(u)
    assert d / e["eps"][0] > 10.0  # rho(d / eps~) = 1 to double precision
    ref = np.empty(C)
    for ch in range(C):
        if ch < G:
            ref[ch] = u @ _torch_bf16(S[ch].astype(np.float32)) / (4 * math.pi * d ** 3)
        else:
            ref[ch] = _torch_bf16(np.array([Sm[ch]], np.float32))[0] / (4 * math.pi * d ** 2)
    np.testing.assert_allclose(y[0], ref, rtol=1e-12, atol=0)
    # and the double moments differ from it by at most the bf16 rounding
    T.update(mu, geometry_channels=G)
    y64 = T.forward(x, 2.0)
    assert np.all(np.abs(y64[0] - y[0]) <= 2.0 ** -8 * np.abs(y64[0]) * 3 + 1e-30)
    assert np.any(y64[0] != y[0])



@pytest.mark.parametrize("m,amb", [(1.0 + 2.0 ** -8, 2.0 ** -7), (1.25, 0.0), (1.0 + 2.0 ** -9, 0.0)])
def test_rounding_ambiguity_allowance(m, amb):
    """One point at the origin, A = 1, n = (1, 0, 0), attribute m: the root is a
    leaf of radius 0, so every other query takes it as far, and its one sum is
    S = m.  m = 1 + 2^-8 is a bf16 tie (the even neighbour 1 is taken): an
    implementation summing in float could have landed on either side, so the
    forward at x = (-10, 0, 0) reports |v_x| 2^-7 with v_x = 10 / (4 pi 10^3);
    a value on a bf16 number (1.25) or far from a boundary reports 0."""
    pts = np.zeros((1, 3), np.float32)
    nrm = np.array([[1.0, 0.0, 0.0]], np.float32)
    T = oracle.Tree(pts, nrm, np.ones(1, np.float32), np.full(1, 1e-3, np.float32))
    T.update(np.array([[m]], np.float32), bf16_moments=True)
    y, allow = T.forward_bf16_allowance(np.array([[-10.0, 0.0, 0.0]], np.float32), 2.0)
    vx = 10.0 / (4 * math.pi * 1e3)
    np.testing.assert_allclose(allow[0, 0], vx * amb, rtol=1e-12, atol=0)
    np.testing.assert_allclose(y[0, 0], vx * _torch_bf16(np.array([m], np.float32))[0], rtol=1e-12)
