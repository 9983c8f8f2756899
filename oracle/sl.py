"""Semi-Lagrangian finite-difference update: characteristic feet, the local entry evaluator
on an HT tensor, and the dense full-tensor SL step used as brute force (Sec. 3.1).

Test infrastructure: part of the FP64 oracle, never called by the CUDA path.

Readings of the paper taken here:

* The frozen-field advection of one RKEI stage is d_t f + v . grad_x f - E(x) . grad_v f = 0
  (electron charge -1, Eq. Vlasov with q_e/m_e = -1).  Its characteristics are
  dx/dt = v, dv/dt = -E(x); the backward foot therefore has v* = v + E tau to first order.
* The paper only says "a high-order RK integrator".  The foot is traced with Kutta's
  third-order Runge-Kutta method on the backward system dz/ds = (-v, E(x)) over s in
  [0, tau], in one step.  E at off-grid points is the tensor-product quadratic
  interpolant of the grid field (the same weights as the update).  ``foot="euler"``
  selects the first-order foot (x - v tau, v + E(x) tau).
* The arithmetic of the foot and of the field interpolation is written as an explicit
  sequence of scalar operations (no fused multiply-add, fixed summation order) so that
  the cell choice floor((y - a)/Delta) is reproducible.
* Higher-order interpolation (the remark after Eq. tp_interp): a grid of interpolation
  order 4 replaces the quadratic weights by the quartic centred Lagrange weights on the
  five-point stencil {j-2, ..., j+2} everywhere the quadratic ones are used -- the leaf
  gathers, the field interpolation of the foot, and the LoMaC correction -- with the same
  cell rule.  Order 2 is the paper's scheme.
"""
from __future__ import annotations

import itertools
from typing import List, Sequence

import numpy as np

from . import grid
from .ht import HT, contract_tree, spatial_linear_index


class PhaseGrid:
    """Grid description: per dimension (lo, hi, N); dimension order (x1..x_dx, v1..v_dv)."""

    def __init__(self, dx: int, dv: int, N: Sequence[int], lo: Sequence[float], hi: Sequence[float],
                 order: int = 2):
        self.dx, self.dv = dx, dv
        self.N = tuple(int(n) for n in N)
        self.lo = tuple(float(a) for a in lo)
        self.hi = tuple(float(b) for b in hi)
        self.order = int(order)   # interpolation order: 2 (quadratic) or 4 (quartic)

    @property
    def S(self):
        """Points of the 1D stencil."""
        return self.order + 1

    @property
    def d(self):
        return self.dx + self.dv

    @property
    def Nx(self):
        return self.N[: self.dx]

    def centres(self, m: int) -> np.ndarray:
        return grid.centres(self.lo[m], self.hi[m], self.N[m])

    def h(self, m: int) -> float:
        return grid.spacing(self.lo[m], self.hi[m], self.N[m])


def interp_spatial(field: np.ndarray, pts: np.ndarray, g: PhaseGrid) -> np.ndarray:
    """Tensor-product interpolation (the grid's order; quadratic by default) of a periodic
    spatial grid field (flattened, x1 slowest) at points pts (S, dx).  Summation runs over
    the stencil in lexicographic order, accumulating (w_1 ... w_dx) * value."""
    dx = g.dx
    Nx = g.Nx
    F = field.reshape(Nx)
    rows, ws = [], []
    for m in range(dx):
        j, xi = grid.locate(pts[:, m], g.lo[m], g.hi[m], Nx[m])
        rows.append(grid.stencil_rows(j, Nx[m], g.order))
        ws.append(grid.stencil_weights(xi, g.order))
    acc = np.zeros(pts.shape[0])
    for s in itertools.product(range(g.S), repeat=dx):
        wprod = ws[0][:, s[0]]
        for m in range(1, dx):
            wprod = wprod * ws[m][:, s[m]]
        val = F[tuple(rows[m][:, s[m]] for m in range(dx))]
        acc = acc + wprod * val
    return acc


def trace_feet(idx: np.ndarray, E: np.ndarray, tau: float, g: PhaseGrid, foot: str = "rk3") -> np.ndarray:
    """Backward characteristic feet of the frozen-field advection for grid tuples idx (S, d).

    Returns the foot coordinates (S, d).  See the module docstring for the integrator."""
    idx = np.asarray(idx, dtype=np.int64)
    dx, dv = g.dx, g.dv
    x = np.stack([g.centres(m)[idx[:, m]] for m in range(dx)], axis=1)
    v = np.stack([g.centres(dx + m)[idx[:, dx + m]] for m in range(dv)], axis=1)

    def Eat(pts):
        return np.stack([interp_spatial(E[m], pts, g) for m in range(dx)], axis=1)

    h = float(tau)
    if foot == "euler":
        e1 = Eat(x)
        return np.concatenate([x - v * h, v + e1 * h], axis=1)
    half = h / 2.0
    two_h = 2.0 * h
    sixth = h / 6.0
    # stage 1: k1 = (-v, E(x))
    k1x = -v
    k1v = Eat(x)
    # stage 2 at z + (h/2) k1
    x2 = x + half * k1x
    v2 = v + half * k1v
    k2x = -v2
    k2v = Eat(x2)
    # stage 3 at z - h k1 + 2h k2
    x3 = (x - h * k1x) + two_h * k2x
    v3 = (v - h * k1v) + two_h * k2v
    k3x = -v3
    k3v = Eat(x3)
    xs = x + sixth * ((k1x + 4.0 * k2x) + k3x)
    vs = v + sixth * ((k1v + 4.0 * k2v) + k3v)
    return np.concatenate([xs, vs], axis=1)


def leaf_vectors_at(ht: HT, feet: np.ndarray, g: PhaseGrid) -> List[np.ndarray]:
    """c^(mu) = w(xi^(mu)) U^(mu)_{J_mu}: the interpolant (quadratic, or the grid's order) of
    every leaf basis column at the foot coordinate of dimension mu (Sec. 3.1).  Returns list
    of (S, r_mu)."""
    c = []
    for m in range(ht.d):
        j, xi = grid.locate(feet[:, m], g.lo[m], g.hi[m], g.N[m])
        w = grid.stencil_weights(xi, g.order)
        rows = grid.stencil_rows(j, g.N[m], g.order)
        U = ht.U[m]
        acc = w[:, 0:1] * U[rows[:, 0]]
        for s in range(1, g.S):
            acc = acc + w[:, s:s + 1] * U[rows[:, s]]
        c.append(acc)
    return c


def correction_at(ht: HT, feet: np.ndarray, g: PhaseGrid) -> np.ndarray:
    """Value of the separable LoMaC correction at off-grid feet: each spatial field dC_k is
    interpolated with the tensor-product quadratic weights and each velocity factor with the
    1D weights (interpolation is linear, so this equals interpolating the summed tensor)."""
    corr = ht.corr
    out = np.zeros(feet.shape[0])
    dCi = [interp_spatial(corr.dC[k], feet[:, : g.dx], g) for k in range(corr.dC.shape[0])]
    for k, vecs in corr.terms:
        t = dCi[k].copy()
        for m, vec in enumerate(vecs):
            mu = g.dx + m
            t = t * grid.interp_1d(vec, feet[:, mu], g.lo[mu], g.hi[mu], g.order)
        out = out + t
    return out


def eval_at_feet(ht: HT, feet: np.ndarray, g: PhaseGrid) -> np.ndarray:
    """f(x*) of an HT state at foot points: leaf interpolation, tree contraction, plus the
    separable correction if present (Sec. 3.1, Eq. tp_interp evaluated in HT form)."""
    out = contract_tree(ht, leaf_vectors_at(ht, feet, g))
    if ht.corr is not None:
        out = out + correction_at(ht, feet, g)
    return out


def sl_eval(ht: HT, E: np.ndarray, tau: float, idx: np.ndarray, g: PhaseGrid, foot: str = "rk3") -> np.ndarray:
    """The local SL-FD entry evaluator: F^{n+1}_i = f(x*_i, t^n) (Eq. SL_basic_formulation),
    with the foot of the frozen-field characteristic through grid tuple i."""
    return eval_at_feet(ht, trace_feet(idx, E, tau, g, foot), g)


# ----------------------------------------------------------------------------------------
# brute force: the dense full-tensor SL step (Eq. tp_interp, O(3^d) per point)
# ----------------------------------------------------------------------------------------

def all_tuples(N: Sequence[int]) -> np.ndarray:
    grids = np.meshgrid(*[np.arange(n) for n in N], indexing="ij")
    return np.stack([q.reshape(-1) for q in grids], axis=1)


def dense_interp(F: np.ndarray, feet: np.ndarray, g: PhaseGrid) -> np.ndarray:
    """<F_J, W(xi)>: the full S^d-point tensor-product interpolation (S = 3: quadratic) of a
    dense tensor at the feet (Eq. tp_interp)."""
    d = F.ndim
    rows, ws = [], []
    for m in range(d):
        j, xi = grid.locate(feet[:, m], g.lo[m], g.hi[m], g.N[m])
        rows.append(grid.stencil_rows(j, g.N[m], g.order))
        ws.append(grid.stencil_weights(xi, g.order))
    acc = np.zeros(feet.shape[0])
    for s in itertools.product(range(g.S), repeat=d):
        wprod = np.ones(feet.shape[0])
        for m in range(d):
            wprod = wprod * ws[m][:, s[m]]
        acc = acc + wprod * F[tuple(rows[m][:, s[m]] for m in range(d))]
    return acc


def dense_sl_step(F: np.ndarray, E: np.ndarray, tau: float, g: PhaseGrid, foot: str = "rk3") -> np.ndarray:
    """One full-rank SL step of the frozen-field advection on the dense grid."""
    idx = all_tuples(g.N)
    feet = trace_feet(idx, E, tau, g, foot)
    return dense_interp(F, feet, g).reshape(g.N)


def constant_feet(g: PhaseGrid, a: Sequence[float], tau: float) -> np.ndarray:
    """Feet x - a tau of constant-coefficient advection at every grid point (Thm. uncond_stab)."""
    idx = all_tuples(g.N)
    pts = np.stack([g.centres(m)[idx[:, m]] for m in range(g.d)], axis=1)
    return pts - np.asarray(a, dtype=np.float64)[None, :] * tau
