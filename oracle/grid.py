"""Uniform cell-centred periodic grids, the 1D quadratic Lagrange weights (Sec. 3.1) and
the higher-order centred Lagrange weights of the remark after Eq. tp_interp.

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


def lagrange_weights(xi, order: int):
    """Lagrange interpolation weights of degree `order` (even) on the centred stencil of
    order + 1 nodes at the integer offsets k = -order/2 .. order/2 from the cell centre,
    evaluated at xi: L_k(xi) = prod_{m != k} (xi - m) / (k - m).  The paper uses order 2
    (Eq. 1d_quadratic_interp_weight) and notes that the HT evaluation extends to higher
    orders (remark after Eq. tp_interp); order 4 is the five-point quartic stencil.
    Returns shape (..., order + 1), nodes in increasing k."""
    if order < 2 or order % 2:
        raise ValueError("order must be even and >= 2")
    xi = np.asarray(xi, dtype=np.float64)
    nodes = range(-(order // 2), order // 2 + 1)
    cols = []
    for k in nodes:
        L = np.ones_like(xi)
        for m in nodes:
            if m != k:
                L = L * (xi - m) / (k - m)
        cols.append(L)
    return np.stack(cols, axis=-1)


def stencil_weights(xi, order: int = 2):
    """The weights of an interpolation order: the paper's quadratic formula for order 2,
    the general centred Lagrange weights otherwise."""
    return weights(xi) if order == 2 else lagrange_weights(xi, order)


def stencil_rows(j, n: int, order: int = 2):
    """Periodic stencil row indices (j - order/2, ..., j + order/2) mod N, shape
    (..., order + 1); order 2 gives (j-1, j, j+1)."""
    j = np.asarray(j, dtype=np.int64)
    h = order // 2
    return np.stack([(j + k) % n for k in range(-h, h + 1)], axis=-1)


def interp_1d(values: np.ndarray, y, lo: float, hi: float, order: int = 2):
    """Interpolation of a periodic grid function at points y with the centred stencil of
    the given order (quadratic by default, Sec. 3.1)."""
    n = values.shape[0]
    j, xi = locate(y, lo, hi, n)
    w = stencil_weights(xi, order)
    rows = stencil_rows(j, n, order)
    return (w * values[rows]).sum(axis=-1)
