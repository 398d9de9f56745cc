"""Hockney-Eastwood / cardinal B-spline assignment weights (Section 2.3.2, Eq. w3d).

Reading of the paper: W^(p) is the centred cardinal B-spline of order p -- the p-fold
convolution of the unit box -- a piecewise polynomial of degree p-1 supported on
|t| < p/2, whose Fourier transform at n/N cycles per mesh cell is sinc^p (Eq. Bk).
For odd p the stencil is centred on n = round(x), for even p on n + 1/2 with
n = floor(x) (Eq. w3d); in both cases the p stencil points are exactly the mesh points
m with |x - m| < p/2, i.e. m = m0 + j, j = 0..p-1, m0 = floor(x - p/2) + 1, and the
weight of point m is W(x - m).

Everything here is written once for any array module ``xp`` (numpy or torch) using
plain arithmetic, so that the torch version is differentiable by autograd.

Pins (tests/test_oracle_bspline.py): partition of unity, zero first moment, vanishing
derivative sum, symmetry, the textbook NGP / CIC / TSC closed forms for p = 1, 2, 3,
the Fourier transform sinc^p by quadrature, and derivatives against central
differences. Parity: pinned.
"""
from __future__ import annotations

import math

import numpy as np


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _indicator(y):
    """1 on [0, 1), 0 elsewhere, with the dtype of y (no gradient)."""
    m = (y >= 0) & (y < 1)
    if _is_torch(y):
        return m.to(y.dtype)
    return m.astype(y.dtype)


def uncentred(p: int, y, deriv: int = 0):
    """N_p(y): uncentred cardinal B-spline on [0, p], or its ``deriv``-th derivative.

    N_1 is the indicator of [0, 1); N_k(y) = (y N_{k-1}(y) + (k - y) N_{k-1}(y - 1))/(k-1);
    d/dy N_k(y) = N_{k-1}(y) - N_{k-1}(y - 1).
    """
    if deriv > 0:
        if p == 1:
            return y * 0.0
        return uncentred(p - 1, y, deriv - 1) - uncentred(p - 1, y - 1.0, deriv - 1)
    if p == 1:
        return _indicator(y)
    return (y * uncentred(p - 1, y) + (p - y) * uncentred(p - 1, y - 1.0)) / (p - 1)


def W(p: int, t, deriv: int = 0):
    """Centred assignment function W^(p)(t) = N_p(t + p/2) and its derivatives in t."""
    return uncentred(p, t + 0.5 * p, deriv)


def stencil_base(p: int, x):
    """First stencil index m0 = floor(x - p/2) + 1 (integer array, same module as x)."""
    if _is_torch(x):
        import torch
        return torch.floor(x.detach() - 0.5 * p).to(torch.int64) + 1
    return np.floor(x - 0.5 * p).astype(np.int64) + 1


def stencil_weights(p: int, x, deriv: int = 0):
    """Weights of the p stencil points m0 + j of mesh coordinate(s) x.

    Returns (m0, w) with w[..., j] = d^deriv/dx^deriv W^(p)(x - (m0 + j)).
    For torch inputs w is differentiable in x.
    """
    m0 = stencil_base(p, x)
    if _is_torch(x):
        import torch
        j = torch.arange(p, dtype=x.dtype)
        t = x[..., None] - (m0[..., None].to(x.dtype) + j)
    else:
        j = np.arange(p, dtype=np.float64)
        t = x[..., None] - (m0[..., None] + j)
    return m0, W(p, t, deriv)


def sinc_response(p: int, n, N):
    """Assignment response sinc^p(n/N) of Eq. Bk for one dimension (numpy, float64)."""
    u = np.asarray(n, dtype=np.float64) / N
    return np.sinc(u) ** p


def closed_form(p: int, t):
    """Textbook low-order assignment functions (Hockney & Eastwood): NGP, CIC, TSC."""
    a = np.abs(np.asarray(t, dtype=np.float64))
    if p == 1:
        return np.where(a < 0.5, 1.0, 0.0)
    if p == 2:
        return np.where(a < 1.0, 1.0 - a, 0.0)
    if p == 3:
        return np.where(a < 0.5, 0.75 - a * a, np.where(a < 1.5, 0.5 * (1.5 - a) ** 2, 0.0))
    raise ValueError(p)


def fourier_transform(p: int, f: float, npts: int = 200001) -> float:
    """Continuous Fourier transform of W^(p) at frequency f (cycles per mesh unit), by
    midpoint quadrature over its support."""
    h = p / npts
    t = -p / 2 + h * (np.arange(npts) + 0.5)      # midpoint rule
    return float(h * np.sum(W(p, t) * np.cos(2 * math.pi * f * t)))
