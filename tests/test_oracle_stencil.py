"""Pins of the higher-order interpolation option (remark after Eq. tp_interp): the quartic
centred Lagrange stencil {j-2, ..., j+2} in the oracle's grid, SL evaluator and dense step.

What fixes it independently of the oracle's own formula:
* the classical midpoint weights of quartic interpolation, (3, -20, 90, 60, -5) / 128 at
  xi = 1/2 (the textbook five-point midpoint rule), the unit vector at xi = 0;
* exact reproduction of polynomials of degree <= 4 and, for x^5, the interpolation error
  equal to the nodal polynomial (xi+2)(xi+1) xi (xi-1)(xi-2) (Lagrange remainder with
  f^(5)/5! = 1);
* fifth-order convergence of the interpolant of a smooth periodic function;
* the 1D von Neumann factor of the SL step bounded by one (the stability property the
  paper proves for the quadratic stencil, Thm. uncond_stab), the l2 norm of a dense step not
  growing, and exact shifts when the displacement is a whole number of cells;
* the HT entry evaluator at order 4 equal to the dense S^d-point interpolation (Eq.
  tp_interp with the quartic weights).
"""
import numpy as np
import pytest

from oracle import grid, sl
from oracle import ht as htmod
from paper_2606_29027_b300 import inputs


def test_quartic_midpoint_and_centre_weights():
    w = grid.lagrange_weights(np.array([0.5, -0.5, 0.0]), 4)
    assert np.allclose(w[0], np.array([3, -20, 90, 60, -5]) / 128.0, rtol=0, atol=1e-15)
    assert np.allclose(w[1], np.array([-5, 60, 90, -20, 3]) / 128.0, rtol=0, atol=1e-15)
    assert np.array_equal(w[2], np.array([0.0, 0.0, 1.0, 0.0, 0.0]))


def test_general_order_two_is_the_papers_quadratic():
    xi = np.random.default_rng(1).uniform(-0.5, 0.5, 200)
    assert np.abs(grid.lagrange_weights(xi, 2) - grid.weights(xi)).max() < 1e-15


def test_quartic_reproduces_degree_four_and_x5_error_is_nodal():
    rng = np.random.default_rng(2)
    xi = rng.uniform(-0.5, 0.5, 300)
    w = grid.lagrange_weights(xi, 4)
    k = np.arange(-2, 3, dtype=np.float64)
    for p in range(5):
        assert np.abs(w @ k ** p - xi ** p).max() < 1e-14, p
    nodal = (xi + 2) * (xi + 1) * xi * (xi - 1) * (xi - 2)
    assert np.abs((xi ** 5 - w @ k ** 5) - nodal).max() < 1e-13
    assert np.abs(nodal).max() > 0.1   # degree 5 is not reproduced


def test_quartic_interpolation_converges_at_fifth_order():
    rng = np.random.default_rng(3)
    y = rng.uniform(0.0, 2 * np.pi, 500)
    errs = []
    for n in (16, 32, 64):
        vals = np.sin(grid.centres(0.0, 2 * np.pi, n) * 3.0)
        errs.append(np.abs(grid.interp_1d(vals, y, 0.0, 2 * np.pi, order=4) - np.sin(3 * y)).max())
    rates = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(24.0 <= r <= 40.0 for r in rates), rates


@pytest.mark.parametrize("order", [2, 4])
def test_von_neumann_factor_bounded(order):
    """1D SL step of constant advection by a displacement (m - xi) cells: the Fourier mode
    e^{i j zeta} is multiplied by e^{-i m zeta} sum_k w_k(xi) e^{i k zeta}; its modulus
    stays at most one for every xi in [-1/2, 1/2] and zeta."""
    xi = np.linspace(-0.5, 0.5, 201)
    zeta = np.linspace(0.0, np.pi, 401)
    w = grid.stencil_weights(xi, order)
    h = order // 2
    k = np.arange(-h, h + 1)
    g = w @ np.exp(1j * np.outer(k, zeta))
    assert np.abs(g).max() <= 1.0 + 1e-14
    assert np.abs(g[:, 0] - 1.0).max() < 1e-14    # constants are kept


def _grid2(order, N=(12, 16)):
    return sl.PhaseGrid(1, 1, N, (0.0, -4.0), (2 * np.pi, 4.0), order=order)


def test_dense_quartic_step_l2_nonincreasing_and_integer_shift_exact():
    g = _grid2(4)
    rng = np.random.default_rng(4)
    F = rng.standard_normal(g.N)
    a = (0.37 * g.h(0) / 0.9, -1.3 * g.h(1) / 0.9)
    G = sl.dense_interp(F, sl.constant_feet(g, a, 0.9), g).reshape(g.N)
    assert np.linalg.norm(G) <= np.linalg.norm(F) * (1 + 1e-14)
    # whole-cell displacement (2, -3) cells: an exact roll of the grid function
    a = (2 * g.h(0), -3 * g.h(1))
    G = sl.dense_interp(F, sl.constant_feet(g, a, 1.0), g).reshape(g.N)
    assert np.abs(G - np.roll(F, (2, -3), axis=(0, 1))).max() < 1e-13


@pytest.mark.parametrize("dims", [(1, 1), (2, 2)])
def test_ht_entries_equal_dense_quartic_interpolation(dims):
    dx, dv = dims
    N = (10, 12) if dx == 1 else (8, 8, 10, 10)
    lo = (0.0,) * dx + (-5.0,) * dv
    hi = (4 * np.pi,) * dx + (5.0,) * dv
    g = sl.PhaseGrid(dx, dv, N, lo, hi, order=4)
    ranks = (3, 4) if dx == 1 else (3, 4, 3, 4, 5, 4)
    h = htmod.from_raw(inputs.random_ht(N, ranks, 5))
    E = inputs.random_field(N[:dx], dx, 0.4, seed=6)
    idx = inputs.random_tuples(N, 200, seed=7)
    got = sl.sl_eval(h, E, 0.8, idx, g)
    feet = sl.trace_feet(idx, E, 0.8, g)
    want = sl.dense_interp(htmod.densify(h), feet, g)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    # and the quartic entries differ from the quadratic ones (the order is in effect)
    g2 = sl.PhaseGrid(dx, dv, N, lo, hi, order=2)
    assert np.abs(sl.sl_eval(h, E, 0.8, idx, g2) - got).max() > 1e-6 * np.abs(want).max()
