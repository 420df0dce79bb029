"""Host-side pieces of the rendering harness (no GPU): the attenuation
coefficient against finite differences of the vacancy (eq. surface_density),
the quadrature weights' telescoping identity, the entropy's extremes and the
shadow-ray samples' geometry."""
import math

import numpy as np
import torch

from paper_2405_16788_gb300 import render


def test_sigma_is_directional_log_derivative_of_vacancy():
    """sigma = |omega . grad v| / v with v = Phi(s (1/2 - D0)): against central
    differences of v along omega for an analytic D0."""
    torch.manual_seed(0)
    a = torch.tensor([1.3, -0.7, 0.4], dtype=torch.float64)
    D0 = lambda x: 0.5 + 0.4 * torch.sin(x @ a)
    gD0 = lambda x: 0.4 * torch.cos(x @ a)[:, None] * a[None, :]
    x = torch.randn(200, 3, dtype=torch.float64)
    om = torch.nn.functional.normalize(torch.randn(200, 3, dtype=torch.float64), dim=1)
    s = 7.0
    v, sigma = render.vacancy_sigma(D0(x), gD0(x), om, s)
    h = 1e-6
    vp = torch.special.ndtr(s * (0.5 - D0(x + h * om)))
    vm = torch.special.ndtr(s * (0.5 - D0(x - h * om)))
    ref = ((vp - vm) / (2 * h)).abs() / v
    assert torch.allclose(sigma, ref, rtol=1e-6, atol=1e-9)


def test_sigma_stays_finite_deep_inside():
    """phi(z)/Phi(z) ~ -z as z -> -infinity (Mills ratio): finite, no 0/0."""
    D0 = torch.tensor([5.0, 20.0, 200.0], dtype=torch.float64)
    g = torch.tensor([[0.0, 0.0, 1.0]] * 3, dtype=torch.float64)
    om = torch.tensor([[0.0, 0.0, 1.0]] * 3, dtype=torch.float64)
    s = 10.0
    _, sigma = render.vacancy_sigma(D0, g, om, s)
    z = s * (0.5 - D0)
    assert torch.all(torch.isfinite(sigma))
    assert torch.allclose(sigma / (s * (-z)), torch.ones(3, dtype=torch.float64), rtol=0.05)


def test_free_flight_weights_telescope():
    """sum_j p_j + T_after = 1 and p_j >= 0 (the standard quadrature)."""
    g = torch.Generator().manual_seed(1)
    sigma = torch.rand(50, 40, generator=g, dtype=torch.float64) * 30
    delta = torch.rand(50, 40, generator=g, dtype=torch.float64) * 0.05
    p, T = render.free_flight(sigma, delta)
    assert torch.all(p >= 0)
    assert torch.allclose(p.sum(1) + T, torch.ones(50, dtype=torch.float64), atol=1e-12)
    # one opaque sample takes all the weight
    sig = torch.zeros(1, 10, dtype=torch.float64)
    sig[0, 3] = 1e6
    p, T = render.free_flight(sig, torch.full((1, 10), 0.1, dtype=torch.float64))
    assert abs(float(p[0, 3]) - 1.0) < 1e-12 and float(T) < 1e-12


def test_entropy_extremes():
    one = torch.zeros(1, 16, dtype=torch.float64)
    one[0, 5] = 1.0
    assert float(render.entropy(one)) == 0.0
    uni = torch.full((1, 16), 1 / 16, dtype=torch.float64)
    assert abs(float(render.entropy(uni)) - math.log(16)) < 1e-12


def test_shadow_samples_lie_on_the_segment_inside_the_clip_sphere():
    g = torch.Generator().manual_seed(2)
    xs = (torch.rand(100, 3, generator=g, dtype=torch.float64) - 0.5) * 1.6
    light = torch.tensor([1.8, 1.2, 2.2], dtype=torch.float64)
    jit = torch.rand(100, 64, generator=g, dtype=torch.float64)
    X, w, d = render.shadow_samples(xs, light, jit, offset=0.05, clip_radius=1.5)
    assert X.shape == (100, 64, 3)
    assert torch.allclose(w.norm(dim=1), torch.ones(100, dtype=torch.float64))
    assert torch.all(d > 0)
    r = X - xs[:, None, :]
    # on the ray toward the light, at increasing distance, inside the clip sphere
    assert torch.allclose(torch.cross(r, w[:, None, :].expand_as(r), dim=-1).norm(dim=-1),
                          torch.zeros(100, 64, dtype=torch.float64), atol=1e-12)
    along = (r * w[:, None, :]).sum(-1)
    assert torch.all(along[:, 1:] > along[:, :-1]) and torch.all(along >= 0.05)
    assert torch.all(X.norm(dim=-1) <= 1.5 + 1e-9)


def test_direct_light_is_lambertian_and_clamped():
    xs = torch.zeros(2, 3, dtype=torch.float64)
    light = torch.tensor([0.0, 0.0, 2.0], dtype=torch.float64)
    gD0 = torch.tensor([[0.0, 0.0, -1.0], [0.0, 0.0, 1.0]], dtype=torch.float64)  # n^ = +z, -z
    albedo = torch.ones(2, 3, dtype=torch.float64)
    T = torch.tensor([0.5, 0.5], dtype=torch.float64)
    out = render.direct_light(albedo, T, gD0, xs, light)
    assert torch.allclose(out[0], torch.full((3,), 0.5 / 4.0, dtype=torch.float64))
    assert torch.all(out[1] == 0.0)
