"""Pin of the oracle's electric-field energy flux (Eq. electric_field_flux) against the local
field-energy balance derived in Supp. A:

    d_t (|E|^2 / 2) = -div F_ep - J . E,     F_ep = -phi grad(d_t phi) + J phi,

with -Lap(phi) = rho, E = -grad(phi), -Lap(d_t phi) = -div J, for any charge density and
current obeying continuity d_t rho + div J = 0.  On a periodic grid whose fields hold only
wavenumbers below a quarter of the grid, products of two fields do not alias, so the spectral
operators satisfy the product rule exactly and the balance holds to rounding.

The time derivative comes from an eighth-order central difference of |E(t)|^2 / 2 over a
prescribed, exactly continuity-preserving path (rho(t), J(t)); nothing of the flux formula
is retyped here.  A planted sign flip of either term of F_ep, or of the source of d_t phi,
breaks the balance by O(1) and is caught.
"""
import math

import numpy as np
import pytest

from oracle import field, macro, sl


def _grid(dx, n, L):
    N = (n,) * dx + (8,) * dx
    lo = (0.0,) * dx + (-4.0,) * dx
    hi = (L,) * dx + (4.0,) * dx
    return sl.PhaseGrid(dx, dx, N, lo, hi)


def _lowmode_field(g, rng, mmax=2):
    """A real periodic field made of wavenumbers |m_i| <= mmax in every spatial dimension."""
    xs = [g.centres(a) for a in range(g.dx)]
    X = np.meshgrid(*xs, indexing="ij")
    out = np.zeros(X[0].shape)
    modes = [m for m in np.ndindex(*(2 * mmax + 1,) * g.dx)]
    for mm in modes:
        m = [q - mmax for q in mm]
        if all(q == 0 for q in m):
            continue
        ph = sum(2 * math.pi * m[a] * X[a] / (g.hi[a] - g.lo[a]) for a in range(g.dx))
        out += rng.standard_normal() * np.cos(ph) + rng.standard_normal() * np.sin(ph)
    return out.reshape(-1)


class Path:
    """rho(t) = rho0 - div(a) sin(w t)/w + div(b) (cos(w t) - 1)/w and
    J(t) = a cos(w t) + b sin(w t): then d_t rho = -div J exactly (spectral div is linear,
    and the mean parts of a and b have no divergence)."""

    def __init__(self, g, seed, w=1.3, n_i=1.0):
        rng = np.random.default_rng(seed)
        self.g, self.w, self.n_i = g, w, n_i
        self.rho0 = 0.1 * _lowmode_field(g, rng)
        # a mean current too: in one dimension F_ep reduces to phi <J>, which a zero-mean
        # current would make vanish
        self.a = np.stack([0.1 * _lowmode_field(g, rng) + 0.05 * rng.standard_normal() for _ in range(g.dx)])
        self.b = np.stack([0.1 * _lowmode_field(g, rng) + 0.05 * rng.standard_normal() for _ in range(g.dx)])
        self.da = field.div(self.a, g)
        self.db = field.div(self.b, g)

    def rho(self, t):
        w = self.w
        return self.rho0 - self.da * math.sin(w * t) / w + self.db * (math.cos(w * t) - 1.0) / w

    def J(self, t):
        return self.a * math.cos(self.w * t) + self.b * math.sin(self.w * t)

    def U(self, t):
        """Conserved variables with rho = n_i - U0 and J = -U1 (the energy row is not used)."""
        g = self.g
        U = np.zeros((g.dv + 2, int(np.prod(g.Nx))))
        U[0] = self.n_i - self.rho(t)
        U[1:1 + g.dv] = -self.J(t)
        return U


def _ep(path, t):
    _, E, _ = field.poisson_field(path.rho(t), path.g)
    return 0.5 * np.sum(E * E, axis=0)


def _dt_ep(path, t, h=2e-2):
    """Eighth-order central difference (coefficients of the Taylor-exact stencil)."""
    c = [4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0]
    s = 0.0
    for k, ck in enumerate(c, start=1):
        s = s + ck * (_ep(path, t + k * h) - _ep(path, t - k * h))
    return s / h


def balance_residual(path, t, flux_fn=None):
    """max |d_t e_p + div F_ep + J.E| relative to max |d_t e_p|."""
    g = path.g
    flux_fn = flux_fn or macro.field_energy_flux
    Fep, E = flux_fn(path.U(t), g, path.n_i)
    J = path.J(t)
    lhs = _dt_ep(path, t)
    res = lhs + field.div(Fep, g) + np.sum(J * E, axis=0)
    return float(np.max(np.abs(res)) / np.max(np.abs(lhs)))


CASES = [(1, 32, 4 * math.pi), (2, 16, 4 * math.pi), (2, 32, 10 * math.pi)]


@pytest.mark.parametrize("dx,n,L", CASES)
@pytest.mark.parametrize("t", [0.0, 0.7])
def test_field_energy_balance_holds(dx, n, L, t):
    path = Path(_grid(dx, n, L), seed=10 * dx + n)
    assert balance_residual(path, t) < 1e-9


def _phi_and_dtphi(U, g, n_i):
    phi = field.solve_poisson(n_i - U[0], g)
    J = -U[1:1 + g.dv]
    dtphi = field.solve_poisson(-field.div(J, g), g)
    return phi, J, dtphi


@pytest.mark.parametrize("dx,n,L", CASES)
@pytest.mark.parametrize("plant", ["J_phi_sign", "phi_grad_dtphi_sign", "current_sign"])
def test_planted_flux_mistakes_are_caught(dx, n, L, plant):
    """Mistakes planted in the oracle's flux break the balance: the sign of J phi, the sign of
    phi grad(d_t phi) (equivalently of the source of the d_t phi Poisson problem), and the
    current taken as +U1 instead of -U1 (which flips J and d_t phi, hence all of F_ep)."""
    g = _grid(dx, n, L)
    path = Path(g, seed=10 * dx + n)
    orig = macro.field_energy_flux

    def planted(U, gg, n_i):
        Fep, E = orig(U, gg, n_i)
        phi, J, dtphi = _phi_and_dtphi(U, gg, n_i)
        if plant == "J_phi_sign":
            return Fep - 2.0 * J * phi, E
        if plant == "phi_grad_dtphi_sign":
            grad = np.stack([field.deriv(dtphi, gg, a) for a in range(gg.dx)])
            return Fep + 2.0 * phi * grad, E
        return -Fep, E

    assert balance_residual(path, 0.7, planted) > 1e-2


def test_K_energy_row_uses_the_flux():
    """Wiring: the energy row of K(U) contains exactly -div F_ep of field_energy_flux (and
    the other rows do not depend on it): replacing the flux by zero changes K by div F_ep in
    the energy row only."""
    from oracle import lomac
    from oracle import ht as htmod

    dx = 1
    g = _grid(dx, 32, 4 * math.pi)
    rng = np.random.default_rng(3)
    x = g.centres(0)
    v = g.centres(1)
    F = htmod.truncate(htmod.from_terms([[1.0 + 0.1 * np.cos(0.5 * x),
                                          np.exp(-v * v / 2) / math.sqrt(2 * math.pi)]]), 1e-12, 8)
    n_i = float(np.mean(field.moments(F, g)[0]))
    cl = macro.make_closure(F, g, n_i)
    U = lomac.conserved_from_moments(field.moments(F, g), g, n_i)
    U = U + 0.01 * rng.standard_normal(U.shape)
    K1 = macro.K_operator(U, cl)
    Fep, _ = macro.field_energy_flux(U, g, n_i)
    orig = macro.field_energy_flux
    try:
        macro.field_energy_flux = lambda UU, gg, ni: (np.zeros_like(orig(UU, gg, ni)[0]), orig(UU, gg, ni)[1])
        K0 = macro.K_operator(U, cl)
    finally:
        macro.field_energy_flux = orig
    assert np.allclose(K1[:-1], K0[:-1], rtol=0, atol=0)
    assert np.max(np.abs((K0[-1] - K1[-1]) - field.div(Fep, g))) < 1e-13 * max(1.0, np.max(np.abs(Fep)))
