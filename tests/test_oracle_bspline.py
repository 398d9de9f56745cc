"""Pins for the oracle's assignment functions (Section 2.3.2, Eqs. w3d and Bk)."""
import math

import numpy as np
import pytest
import torch

from oracle import bspline

ORDERS = [1, 2, 3, 4, 5, 6, 7]


@pytest.mark.parametrize("p", ORDERS)
def test_partition_of_unity_and_moments(p):
    rng = np.random.default_rng(p)
    x = rng.uniform(-50, 50, size=500)
    m0, w = bspline.stencil_weights(p, x)
    _, dw = bspline.stencil_weights(p, x, 1)
    m = m0[:, None] + np.arange(p)
    assert np.allclose(w.sum(1), 1.0, atol=1e-13)
    # every stencil point satisfies |x - m| < p/2 and weights are non-negative
    assert np.all(np.abs(x[:, None] - m) <= p / 2 + 1e-12)
    assert np.all(w >= -1e-15)
    if p >= 2:
        # first moment vanishes (the assignment preserves the centre of charge)
        assert np.allclose((w * (x[:, None] - m)).sum(1), 0.0, atol=1e-12)
        # derivative weights sum to zero (d/dx of the partition of unity)
        assert np.allclose(dw.sum(1), 0.0, atol=1e-12)


@pytest.mark.parametrize("p", ORDERS)
def test_symmetry_and_support(p):
    t = np.linspace(-p / 2 - 1, p / 2 + 1, 2001)
    w = bspline.W(p, t)
    assert np.allclose(w, bspline.W(p, -t), atol=1e-14) or p == 1
    assert np.all(w[np.abs(t) >= p / 2] == 0.0)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_textbook_closed_forms(p):
    # NGP, CIC and TSC of Hockney & Eastwood
    t = np.linspace(-2, 2, 4001)
    t = t[np.abs(np.abs(t) - 0.5) > 1e-9]
    assert np.allclose(bspline.W(p, t), bspline.closed_form(p, t), atol=1e-14)


@pytest.mark.parametrize("p", ORDERS)
def test_fourier_transform_is_sinc_power(p):
    # the continuous transform at f cycles per mesh cell is sinc^p(f): Eq. Bk
    for f in (0.0, 0.13, 0.37, 0.5):
        ft = bspline.fourier_transform(p, f)
        assert abs(ft - np.sinc(f) ** p) < 2e-6


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("deriv", [1, 2, 3])
def test_derivatives_central_differences(p, deriv):
    if deriv >= p:
        pytest.skip("derivative is a sum of deltas")
    rng = np.random.default_rng(10 * p + deriv)
    t = rng.uniform(-p / 2, p / 2, size=200)
    # stay away from the knots where this derivative order is discontinuous
    frac = np.abs((t + p / 2) - np.round(t + p / 2))
    t = t[frac > 1e-3]
    h = 1e-5
    fd = (bspline.W(p, t + h, deriv - 1) - bspline.W(p, t - h, deriv - 1)) / (2 * h)
    assert np.allclose(bspline.W(p, t, deriv), fd, atol=1e-6 * p ** deriv)


@pytest.mark.parametrize("p", [3, 4, 6])
def test_torch_autograd_matches_analytic_derivative(p):
    x = torch.tensor(np.random.default_rng(1).uniform(0, 30, size=64), dtype=torch.float64,
                     requires_grad=True)
    _, w = bspline.stencil_weights(p, x)
    g = torch.autograd.grad(w.sum(1).sum(), x)[0]     # partition of unity => zero
    assert torch.allclose(g, torch.zeros_like(g), atol=1e-12)
    _, w = bspline.stencil_weights(p, x)
    _, dw = bspline.stencil_weights(p, x.detach(), 1)
    gj = torch.autograd.grad(w[:, 1].sum(), x)[0]
    assert torch.allclose(gj, dw[:, 1], atol=1e-12)


def test_stencil_origin_matches_paper_rule():
    # odd p: centred on n = round(x); even p: centred on floor(x) + 1/2 (Eq. w3d)
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 40, size=1000)
    for p in ORDERS:
        m0 = bspline.stencil_base(p, x)
        if p % 2:
            n = np.floor(x + 0.5)
            assert np.all(m0 == n - (p - 1) // 2)
        else:
            n = np.floor(x)
            assert np.all(m0 == n - p // 2 + 1)
