"""Uniform cell-centred periodic grids and the 1D quadratic Lagrange weights (Sec. 3.1).

Test infrastructure: part of the FP64 oracle, never called by the CUDA path.
"""
from __future__ import annotations

import numpy as np


def spacing(lo: float, hi: float, n: int) -> float:
    """Mesh width Delta = (b - a) / N of a uniform grid on [a, b] (Sec. 3.1)."""
    return (hi - lo) / n


def centres(lo: float, hi: float, n: int) -> np.ndarray:
    """Cell centres x_i = a + (i + 1/2) Delta, i = 0..N-1 (0-based form of Sec. 3.1)."""
    h = spacing(lo, hi, n)
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * h


def locate(y, lo: float, hi: float, n: int):
    """Cell containing a foot y and its normalised offset (Sec. 3.1).

    The foot lies in cell I_j = [a + j Delta, a + (j+1) Delta] with j = floor((y - a)/Delta);
    xi = (y - x_j) / Delta in [-1/2, 1/2).  At a cell face (xi = -1/2 exactly) the floor
    rule takes the cell on the right; the paper's analysis uses the open interval, and the
    two stencils agree to O(Delta^3).  The grid is periodic in every direction, so the
    stencil rows are taken modulo N by the caller.
    Returns (j, xi) with j not yet wrapped.
    """
    h = spacing(lo, hi, n)
    t = (np.asarray(y, dtype=np.float64) - lo) / h
    j = np.floor(t)
    xi = t - j - 0.5
    return j.astype(np.int64), xi


def weights(xi):
    """1D quadratic Lagrange weights on the stencil {j-1, j, j+1} (Eq. 1d_quadratic_interp_weight):
    w(xi) = ( xi (xi - 1) / 2,  1 - xi^2,  xi (xi + 1) / 2 ).  Returns shape (..., 3)."""
    xi = np.asarray(xi, dtype=np.float64)
    w0 = 0.5 * xi * (xi - 1.0)
    w1 = 1.0 - xi * xi
    w2 = 0.5 * xi * (xi + 1.0)
    return np.stack([w0, w1, w2], axis=-1)


def stencil_rows(j, n: int):
    """Periodic stencil row indices (j-1, j, j+1) mod N, shape (..., 3)."""
    j = np.asarray(j, dtype=np.int64)
    return np.stack([(j - 1) % n, j % n, (j + 1) % n], axis=-1)


def interp_1d(values: np.ndarray, y, lo: float, hi: float):
    """Quadratic interpolation of a periodic grid function at points y (Sec. 3.1)."""
    n = values.shape[0]
    j, xi = locate(y, lo, hi, n)
    w = weights(xi)
    rows = stencil_rows(j, n)
    return (w * values[rows]).sum(axis=-1)
