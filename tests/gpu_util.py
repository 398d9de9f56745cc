"""Helpers shared by the GPU parity tests (comparison metrics and frame preparation).

Inputs are rounded to float32 once, and the oracle receives exactly those float32 values
(converted to float64), so oracle and CUDA path see the same input."""
import numpy as np


def f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def relmax(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def relrmse(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.sqrt(np.mean((a - b) ** 2)) / max(np.sqrt(np.mean(b ** 2)), 1e-300))


def sym6(H):
    """[n,3,3] -> [n,6] in the order xx, yy, zz, xy, xz, yz."""
    return np.stack([H[:, 0, 0], H[:, 1, 1], H[:, 2, 2], H[:, 0, 1], H[:, 0, 2], H[:, 1, 2]], 1)


def prepared(frame):
    """(pos, q, mu) rounded to float32 and returned as float64 arrays."""
    return f32(frame.pos), f32(frame.q), f32(frame.mu)


# Tolerances. The energy and force bars are the ones stated for float32 mesh work against
# the float64 plain PME on the same mesh (relative energy 1e-6, relative force RMSE 1e-5).
# Intermediate mesh quantities are held to a max-norm bar of the same order. The backward
# (a Hessian-vector product) sums terms of both signs whose magnitudes exceed the result by
# up to ~10x on top of the float32 gradient error, so its RMSE bar is 1e-4.
TOL_E = 1e-6
TOL_F = 1e-5
TOL_MESH = 2e-5
TOL_HVP = 1e-4
