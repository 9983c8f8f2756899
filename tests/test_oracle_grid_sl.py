"""Oracle pins: grid, weights, the SL-FD update and its stability (Sec. 3.1; Appendix A)."""
import math
import os

import numpy as np
import pytest

from oracle import grid, sl
from oracle import ht as htmod
from paper_2606_29027_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_weights_partition_of_unity_and_quadratics():
    xi = np.linspace(-0.5, 0.4999, 101)
    w = grid.weights(xi)
    assert np.allclose(w.sum(axis=1), 1.0, atol=1e-15)
    # quadratic polynomials are reproduced exactly on the stencil nodes -1, 0, 1
    nodes = np.array([-1.0, 0.0, 1.0])
    for p in ([1, 0, 0], [0, 1, 0], [0, 0, 1], [0.3, -1.7, 2.2]):
        vals = np.polyval(p, nodes)
        assert np.allclose(w @ vals, np.polyval(p, xi), atol=1e-14)
    # w(0) selects the centre, w(+-1) the neighbours (Lagrange property)
    assert np.allclose(grid.weights(0.0), [0, 1, 0])
    assert np.allclose(grid.weights(1.0), [0, 0, 1])
    assert np.allclose(grid.weights(-1.0), [1, 0, 0])


def test_golden_grid_points():
    with open(os.path.join(GOLDEN, "grid_points.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        lo, hi, n, i1, val = float(r[0]), float(r[1]), int(r[2]), int(r[3]), float(r[4])
        assert grid.centres(lo, hi, n)[i1 - 1] == pytest.approx(val, abs=1e-14)


def test_locate_periodic():
    j, xi = grid.locate(np.array([0.01, 0.99, 1.51, -0.26]), 0.0, 1.0, 2)
    assert list(j) == [0, 1, 3, -1]
    assert np.allclose(xi, [0.02 - 0.5, 1.98 - 1.5, 3.02 - 3.5, -0.52 + 1 - 0.5])
    assert list(grid.stencil_rows(np.array([-1, 3]), 2)[0]) == [0, 1, 0]


def _g1d(lam, zeta):
    return 1.0 + lam ** 2 * (math.cos(zeta) - 1.0) - 1j * lam * math.sin(zeta)


def _advect_mode(N, L, a, tau, m):
    """Apply the dense SL step to the real and imaginary parts of one Fourier mode."""
    g = sl.PhaseGrid(1, 0, (N,), (0.0,), (L,))
    x = g.centres(0)
    feet = sl.constant_feet(g, (a,), tau)
    kx = 2 * math.pi * m / L
    re = sl.dense_interp(np.cos(kx * x), feet, g)
    im = sl.dense_interp(np.sin(kx * x), feet, g)
    return (re + 1j * im) / np.exp(1j * kx * x)


@pytest.mark.parametrize("lam", [0.0, 0.13, -0.37, 0.49])
@pytest.mark.parametrize("m", [1, 3, 7])
def test_amplification_factor_small_cfl(lam, m):
    """Von Neumann factor g_1D(lambda, zeta) = 1 + lambda^2 (cos zeta - 1) - i lambda sin zeta
    for |lambda| <= 1/2 (Appendix A)."""
    N, L = 32, 2.0
    h = L / N
    ratio = _advect_mode(N, L, a=lam * h / 0.1, tau=0.1, m=m)
    zeta = 2 * math.pi * m / N
    assert np.allclose(ratio, _g1d(lam, zeta), atol=1e-13)


@pytest.mark.parametrize("lam", [1.3, -2.8, 5.2, 17.41])
def test_amplification_factor_large_cfl(lam):
    """Large CFL: g(lambda) = exp(-i m zeta) g(theta), lambda = m + theta (Appendix A)."""
    N, L, mode = 32, 2.0, 3
    h = L / N
    ratio = _advect_mode(N, L, a=lam * h, tau=1.0, m=mode)
    zeta = 2 * math.pi * mode / N
    mm = round(lam)
    theta = lam - mm
    want = np.exp(-1j * mm * zeta) * _g1d(theta, zeta)
    assert np.allclose(ratio, want, atol=1e-12)
    assert np.all(np.abs(ratio) <= 1.0 + 1e-13)


def test_amplification_factorises_in_2d():
    """d-D factor = product of 1D factors (Appendix A, arbitrary dimensions)."""
    N = (16, 12)
    L = (2.0, 3.0)
    g = sl.PhaseGrid(1, 1, N, (0.0, 0.0), L)
    lam = (0.31, -2.2)
    tau = 0.5
    a = [lam[m] * L[m] / N[m] / tau for m in range(2)]
    feet = sl.constant_feet(g, a, tau)
    m1, m2 = 2, 5
    X, Y = np.meshgrid(g.centres(0), g.centres(1), indexing="ij")
    ph = 2 * math.pi * (m1 * X / L[0] + m2 * Y / L[1])
    re = sl.dense_interp(np.cos(ph), feet, g)
    im = sl.dense_interp(np.sin(ph), feet, g)
    ratio = (re + 1j * im).reshape(N) / np.exp(1j * ph)
    want = 1.0
    for m, mode in enumerate((m1, m2)):
        zeta = 2 * math.pi * mode / N[m]
        mm = round(lam[m])
        want = want * np.exp(-1j * mm * zeta) * _g1d(lam[m] - mm, zeta)
    assert np.allclose(ratio, want, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_l2_nonincrease(seed):
    """||F^{n+1}||_2 <= ||F^n||_2 for any dt (Thm. uncond_stab)."""
    rng = np.random.default_rng(seed)
    N = (10, 8, 6)
    g = sl.PhaseGrid(2, 1, N, (0, 0, 0), (1, 2, 3))
    F = rng.standard_normal(N)
    for tau in (0.1, 1.7, 23.0):
        a = rng.standard_normal(3) * 3
        Fn = sl.dense_interp(F, sl.constant_feet(g, a, tau), g).reshape(N)
        assert np.linalg.norm(Fn) <= np.linalg.norm(F) * (1 + 1e-14)


def _rand_state(N, ranks, seed, with_corr):
    h = htmod.from_raw(inputs.random_ht(N, ranks, seed, smooth=False))
    if with_corr:
        d = len(N)
        dx = d // 2
        rng = np.random.default_rng(seed + 100)
        nx = int(np.prod(N[:dx]))
        dv = d - dx
        dC = rng.standard_normal((dv + 2, nx))
        terms = [(k, [rng.standard_normal(N[dx + m]) for m in range(dv)]) for k in range(dv + 2)]
        h.corr = htmod.Correction(dC=dC, terms=terms)
    return h


@pytest.mark.parametrize("case", [
    ((16, 32), (4, 5), "rk3"), ((16, 32), (4, 5), "euler"),
    ((8, 8, 8, 8), (3, 4, 2, 3, 5, 4), "rk3"), ((12, 12, 12, 12), (6, 5, 6, 4, 6, 6), "rk3")])
@pytest.mark.parametrize("with_corr", [False, True])
def test_ht_entry_evaluator_equals_full_tensor_interpolation(case, with_corr):
    """sl_eval on the HT (leaf interpolation + tree contraction) equals the full 3^d-point
    tensor-product interpolation of the densified tensor at every grid point (Sec. 3.1)."""
    N, ranks, foot = case
    d = len(N)
    dx = d // 2
    lo = (0.0,) * dx + (-6.0,) * dx
    hi = (4 * math.pi,) * dx + (6.0,) * dx
    g = sl.PhaseGrid(dx, d - dx, N, lo, hi)
    h = _rand_state(N, ranks, seed=sum(N) + len(ranks), with_corr=with_corr)
    E = inputs.random_field(N[:dx], dx, 0.7, seed=5)
    tau = 0.37
    idx = sl.all_tuples(N)
    got = sl.sl_eval(h, E, tau, idx, g, foot).reshape(N)
    want = sl.dense_sl_step(htmod.densify(h), E, tau, g, foot)
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)


def test_free_streaming_exact_shift():
    """E = 0 with v tau / Delta x integer at every v: the SL step is an exact grid shift,
    i.e. f(x - v t, v) (free streaming)."""
    Nx, Nv = 16, 8
    L = 2 * math.pi
    dxh = L / Nx
    dv = 0.5
    tau = 2 * dxh / dv            # v_k tau / Delta x = 2k - Nv + 1 integer
    g = sl.PhaseGrid(1, 1, (Nx, Nv), (0.0, -dv * Nv / 2), (L, dv * Nv / 2))
    x, v = g.centres(0), g.centres(1)
    F0 = np.outer(1 + 0.3 * np.cos(x) + 0.2 * np.sin(2 * x), np.exp(-v ** 2))
    h = htmod.truncate(htmod.from_terms([[1 + 0.3 * np.cos(x) + 0.2 * np.sin(2 * x), np.exp(-v ** 2)]]), 1e-15, 8)
    E = np.zeros((1, Nx))
    idx = sl.all_tuples((Nx, Nv))
    got = sl.sl_eval(h, E, tau, idx, g).reshape(Nx, Nv)
    shift = np.rint(v * tau / dxh).astype(int)
    want = np.stack([np.roll(F0[:, k], shift[k]) for k in range(Nv)], axis=1)
    assert np.allclose(got, want, atol=1e-14)


def test_free_streaming_third_order():
    """E = 0, generic v tau: one step reproduces f0(x - v tau, v) with O(Delta x^3) error
    (the worst case over many offsets halves 8-fold per grid halving)."""
    errs = []
    taus = np.linspace(0.05, 1.95, 23)
    for Nx in (32, 64, 128):
        L = 2 * math.pi
        g = sl.PhaseGrid(1, 1, (Nx, 4), (0.0, 0.3), (L, 1.3))
        x, v = g.centres(0), g.centres(1)
        f = lambda y: np.exp(np.sin(y))
        h = htmod.from_terms([[f(x), np.ones(4)]])
        idx = sl.all_tuples((Nx, 4))
        e = 0.0
        for tau in taus:
            got = sl.sl_eval(h, np.zeros((1, Nx)), tau, idx, g).reshape(Nx, 4)
            want = f(x[:, None] - v[None, :] * tau)
            e = max(e, np.max(np.abs(got - want)))
        errs.append(e)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.8), rates


def test_rk3_foot_exact_for_uniform_field():
    """A uniform field E0 makes the electron characteristic (dx/dt = v, dv/dt = -E0,
    Eq. Vlasov with q_e/m_e = -1) a quadratic in time; the third-order Runge-Kutta foot is
    then exact: x* = x - v tau - E0 tau^2 / 2, v* = v + E0 tau."""
    N = (16, 16, 8, 8)
    g = sl.PhaseGrid(2, 2, N, (0, 0, -3, -3), (10, 10, 3, 3))
    E0 = (0.7, -0.4)
    E = np.stack([np.full(256, E0[0]), np.full(256, E0[1])])
    idx = inputs.random_tuples(N, 50, seed=3)
    tau = 0.9
    feet = sl.trace_feet(idx, E, tau, g)
    for m in range(2):
        x = g.centres(m)[idx[:, m]]
        v = g.centres(2 + m)[idx[:, 2 + m]]
        assert np.allclose(feet[:, m], x - v * tau - E0[m] * tau ** 2 / 2, atol=1e-13)
        assert np.allclose(feet[:, 2 + m], v + E0[m] * tau, atol=1e-13)
    eul = sl.trace_feet(idx, E, tau, g, foot="euler")
    assert np.allclose(eul[:, 2], g.centres(2)[idx[:, 2]] + E0[0] * tau, atol=1e-13)
