"""Implicit macroscopic update closed by the LoMaC-corrected kinetic state: the residual
G(U), the Jacobian-free Newton-Krylov solve, and the BE / BDF3 / DIRK3 time discretisations
(Sec. 2.2, Eq. macro_sys, macro_sys_comp, electric_field_flux; Sec. 3.2.3,
Eq. BE_macro, BE_nonlinear_system; Sec. 4 solver settings).

Test infrastructure: part of the FP64 oracle, never called by the CUDA path.

Readings:
* D_x is the spectral divergence for every flux component (the paper names a conservative
  flux difference and, for the field terms, spectral differentiation; spectral
  derivatives are exactly conservative and compatible with the field operators).
* The kinetic flux moments of F^{n+1}(U) are those of F* plus sum_k dC_k(U) <psi Q_k>,
  with dC(U) = C~(U) - C(F*) (Eq. LoMaC_update_discrete is linear in R(U)).  The mass flux
  is M1 of F^{n+1}(U), which equals U1 by construction.
* d_t phi solves -Lap(d_t phi) = -div J with J = -U1 (Eq. current_density).
* Newton stops when ||G||_inf <= tol * max(1, ||U^n||_inf); GMRES(m) with relative
  tolerance krylov_tol on the Newton correction; finite-difference Jacobian-vector
  products with h = sqrt(eps_mach) (1 + ||U||_2) / ||v||_2; no preconditioner; initial
  guess U(F*) (Sec. 3.2.3).
* DIRK3 is the three-stage, third-order, S-stable, stiffly accurate method of Alexander
  (1977, Thm. 5); BDF3 is the fixed-step Gear formula.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field as dfield
from typing import Callable, List

import numpy as np

from . import field, lomac
from .ht import HT
from .sl import PhaseGrid

EPS_MACH = 2.0 ** -52

# Alexander (1977) Thm. 5: gamma = root in (1/6, 1/2) of x^3 - 3x^2 + 3x/2 - 1/6.
def _dirk3_gamma():
    x = 0.4358665215
    for _ in range(60):
        f = x ** 3 - 3 * x ** 2 + 1.5 * x - 1.0 / 6.0
        df = 3 * x ** 2 - 6 * x + 1.5
        x -= f / df
    return x

DIRK3_GAMMA = _dirk3_gamma()


def dirk3_tableau():
    """(A, c) of the S-stable stiffly accurate DIRK3 (Alexander 1977, Thm. 5)."""
    g = DIRK3_GAMMA
    b1 = -(6 * g * g - 16 * g + 1) / 4.0
    b2 = (6 * g * g - 20 * g + 5) / 4.0
    A = np.array([[g, 0.0, 0.0], [(1 - g) / 2.0, g, 0.0], [b1, b2, g]])
    c = np.array([g, (1 + g) / 2.0, 1.0])
    return A, c


BDF3 = dict(a=(18.0 / 11.0, -9.0 / 11.0, 2.0 / 11.0), beta=6.0 / 11.0)

# Upper bound on the ratio h_n / h_{n-1} of adjacent steps under which variable-step BDF3 is
# stable (Sec. 3.2.3 defers to the step-ratio analysis of Li and Liao for it; the paper does
# not print the value).  Reading: 1.4877, the bound that analysis states for BDF3.
BDF3_RATIO_MAX = 1.4877


def bdf3_variable(h):
    """Variable-step BDF3 (Gear 1971; Sec. 3.2.3): the cubic through (t_{n+1}, U^{n+1}),
    (t_n, U^n), (t_{n-1}, U^{n-1}), (t_{n-2}, U^{n-2}) is differentiated at t_{n+1} and set equal
    to K(U^{n+1}).  h = (h_n, h_{n-1}, h_{n-2}), the current step first.  Returns (a, beta) with
        U^{n+1} - beta h_n K(U^{n+1}) = a[0] U^n + a[1] U^{n-1} + a[2] U^{n-2}.
    Equal steps give the fixed-step BDF3 table."""
    hn, h1, h2 = (float(x) for x in h)
    t = [0.0, -hn, -hn - h1, -hn - h1 - h2]          # t_{n+1} = 0, then t_n, t_{n-1}, t_{n-2}
    dl = []                                           # Lagrange basis derivatives at t_{n+1}
    for j in range(4):
        if j == 0:
            dl.append(sum(1.0 / (t[0] - t[m]) for m in range(1, 4)))
            continue
        num = 1.0
        den = 1.0
        for m in range(4):
            if m != j:
                den *= t[j] - t[m]
                if m != 0:
                    num *= t[0] - t[m]
        dl.append(num / den)
    beta = 1.0 / (dl[0] * hn)
    return tuple(-dl[j] / dl[0] for j in (1, 2, 3)), beta


@dataclass
class Closure:
    """Everything G needs that comes from F*: its flux moments, C(F*), the LoMaC basis and
    the scalar tables <psi Q_k>."""
    g: PhaseGrid
    n_i: float
    basis: list
    mom_star: np.ndarray        # (n_mom, Nx) moments of F*
    C_star: np.ndarray          # (dv+2, Nx)
    table: np.ndarray           # (n_mom, dv+2)


def make_closure(Fstar: HT, g: PhaseGrid, n_i: float, delta: float = lomac.DELTA_DEFAULT) -> Closure:
    B = lomac.basis_from_ht(Fstar, g, delta)
    mom = field.moments(Fstar, g)
    C = lomac.coefficients_from_moments(mom, B, g)
    return Closure(g=g, n_i=n_i, basis=B, mom_star=mom, C_star=C, table=lomac.flux_tables(B, g))


def K_operator(U: np.ndarray, cl: Closure) -> np.ndarray:
    """K(U) = -D_x . F(U) + S(U): the right-hand side of Eq. macro_sys with the kinetic
    closure of the LoMaC-corrected state and the field-energy flux of
    Eq. electric_field_flux.  U is (dv+2, Nx) = (n, m_1..m_dv, e)."""
    g = cl.g
    dx, dv = g.dx, g.dv
    if dx != dv:
        raise ValueError("Vlasov-Poisson needs dx == dv")
    dC = lomac.coefficients_from_U(U, cl.basis, g, cl.n_i) - cl.C_star
    mom_new = cl.mom_star + cl.table @ dC                 # moments of F^{n+1}(U)
    idx = 1 + dv + 1
    Pi = {}
    for a in range(dv):
        for b in range(a, dv):
            Pi[(a, b)] = Pi[(b, a)] = mom_new[idx]
            idx += 1
    Q3 = [mom_new[idx + a] for a in range(dv)]
    Fep, E = field_energy_flux(U, g, cl.n_i)
    out = np.zeros_like(U)
    # mass: d_t n + div(M1) = 0
    out[0] = -field.div(U[1:1 + dv], g)
    # momentum: d_t m_b + sum_a d_a <v_a v_b f> = rho_e E_b, rho_e = -n
    for b in range(dv):
        flux_b = np.stack([Pi[(a, b)] for a in range(dx)])
        out[1 + b] = -field.div(flux_b, g) + (-U[0]) * E[b]
    # energy: d_t e + div( <|v|^2 v f>/2 - phi grad(d_t phi) + J phi ) = 0
    Fe = np.stack([0.5 * Q3[a] + Fep[a] for a in range(dx)])
    out[1 + dv] = -field.div(Fe, g)
    return out


def field_energy_flux(U: np.ndarray, g: PhaseGrid, n_i: float):
    """The electric-field energy flux F_ep = -phi grad(d_t phi) + J phi of
    Eq. electric_field_flux (epsilon_0 = 1) and the field E, from the conserved variables:
    rho = n_i - U0 (Eq. charge_density), J = -U1 (Eq. current_density), phi and E by the
    spectral Poisson solve, and d_t phi from -Lap(d_t phi) = -div J (Supp. A).  Returns
    (F_ep (dx, Nx), E (dx, Nx))."""
    dx, dv = g.dx, g.dv
    rho = n_i - U[0]
    phi, E, _ = field.poisson_field(rho, g)
    J = -U[1:1 + dv]
    dtphi = field.solve_poisson(-field.div(J, g), g)
    grad_dtphi = [field.deriv(dtphi, g, a) for a in range(dx)]
    Fep = np.stack([-phi * grad_dtphi[a] + J[a] * phi for a in range(dx)])
    return Fep, E


def gmres(Aop: Callable[[np.ndarray], np.ndarray], b: np.ndarray, rtol: float, restart: int,
          maxit: int):
    """Restarted GMRES(m) from x0 = 0 with modified Gram-Schmidt and Givens rotations."""
    n = b.size
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return x, 0
    its = 0
    r = b.copy()
    while its < maxit:
        beta = float(np.linalg.norm(r))
        if beta <= rtol * bnorm:
            break
        m = restart
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        gvec = np.zeros(m + 1)
        gvec[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            w = Aop(V[j])
            its += 1
            for i in range(j + 1):
                H[i, j] = float(w @ V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            j_done = j + 1
            if abs(gvec[j + 1]) <= rtol * bnorm or its >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), gvec[:j_done])
        x = x + V[:j_done].T @ y
        r = b - Aop(x) if its < maxit else r
        if abs(gvec[j_done]) <= rtol * bnorm:
            break
    return x, its


@dataclass
class NewtonStats:
    newton: int = 0
    krylov: int = 0
    residual: float = 0.0
    converged: bool = False
    g_evals: int = 0


def jfnk(Gfun: Callable[[np.ndarray], np.ndarray], U0: np.ndarray, tol_abs: float,
         krylov_tol: float, restart: int = 30, newton_max: int = 20, krylov_max: int = 200):
    """Jacobian-free Newton-Krylov solve of G(U) = 0 (Sec. 3.2.3)."""
    st = NewtonStats()
    U = U0.copy()
    shape = U.shape
    Gu = Gfun(U)
    st.g_evals += 1
    for _ in range(newton_max):
        res = float(np.max(np.abs(Gu)))
        st.residual = res
        if res <= tol_abs:
            st.converged = True
            break
        u = U.reshape(-1)
        g0 = Gu.reshape(-1)
        unorm = float(np.linalg.norm(u))

        def Jv(vv):
            vn = float(np.linalg.norm(vv))
            if vn == 0.0:
                return np.zeros_like(vv)
            h = math.sqrt(EPS_MACH) * (1.0 + unorm) / vn
            st.g_evals += 1
            return (Gfun((u + h * vv).reshape(shape)).reshape(-1) - g0) / h

        delta, its = gmres(Jv, -g0, krylov_tol, restart, krylov_max)
        st.krylov += its
        st.newton += 1
        U = (u + delta).reshape(shape)
        Gu = Gfun(U)
        st.g_evals += 1
    else:
        st.residual = float(np.max(np.abs(Gu)))
        st.converged = st.residual <= tol_abs
    return U, st


def newton_tol_abs(tol: float, Un: np.ndarray) -> float:
    return tol * max(1.0, float(np.max(np.abs(Un))))
