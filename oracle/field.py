"""Velocity moments of a phase-space state and the spectral field solver (Sec. 2, Eq. raw
moments, Eq. charge_density, Eq. Poisson/Efromphi; Sec. 3.2.3 spectral differentiation).

Test infrastructure: part of the FP64 oracle, never called by the CUDA path.

Readings:
* Velocity integrals use the midpoint rule of the cell-centred grid, w^v = prod Delta v
  (Supp. B.1, Eq. inner_global).
* All x-derivatives are spectral (FFT).  The derivative symbol is i k with the Nyquist
  wavenumber of an even grid set to zero, and the Laplacian is the composition
  div(grad) of the same symbols, -sum_m k_m^2; this is what makes the discrete gradient,
  divergence and Laplacian algebraically compatible (Sec. 3.2.3).  Poisson's equation
  -Lap(phi) = rho is inverted on every mode with sum_m k_m^2 > 0; the others get phi = 0.
* The ion density n_i is the mean of M0 of the initial state, so that rho has zero mean.
"""
from __future__ import annotations

import numpy as np

from .ht import HT, Correction
from .sl import PhaseGrid


def moment_monomials(dv: int):
    """The list of velocity weight functions psi(v) of the moments, each as a list of
    (coefficient, exponent-tuple) monomials.  Order:
      M0, M1_1..M1_dv, M2 (Eq. raw moments),
      <v_a v_b f> for a <= b, <|v|^2 v_a f> (flux moments of Eq. macro_sys_comp)."""
    e = [tuple(1 if m == a else 0 for m in range(dv)) for a in range(dv)]
    add = lambda *ts: tuple(sum(t[m] for t in ts) for m in range(dv))
    zero = tuple([0] * dv)
    out = [[(1.0, zero)]]
    out += [[(1.0, e[a])] for a in range(dv)]
    out += [[(1.0, add(e[m], e[m])) for m in range(dv)]]
    for a in range(dv):
        for b in range(a, dv):
            out += [[(1.0, add(e[a], e[b]))]]
    for a in range(dv):
        out += [[(1.0, add(e[m], e[m], e[a])) for m in range(dv)]]
    return out


def n_moments(dv: int) -> int:
    return 1 + dv + 1 + dv * (dv + 1) // 2 + dv


def _leaf_moment_vectors(ht: HT, g: PhaseGrid, expo):
    """sum_j U_mu[j, :] v_j^p Delta v for every velocity leaf (the leaf contraction)."""
    out = []
    for m in range(g.dv):
        mu = g.dx + m
        v = g.centres(mu)
        out.append(ht.U[mu].T @ (v ** expo[m] * g.h(mu)))
    return out


def ht_moment(ht: HT, g: PhaseGrid, psi) -> np.ndarray:
    """Moment <psi f>_v of the HT part as a spatial field (flattened, x1 slowest):
    contract the velocity leaves with psi, then go up the tree (Supp. B.2, Eq. disc_m0..m2)."""
    total = None
    for coef, expo in psi:
        lv = _leaf_moment_vectors(ht, g, expo)
        if g.d == 2:
            fld = ht.U[0] @ (ht.Broot @ lv[0])
        else:
            m34 = np.einsum("ceq,c,e->q", ht.B34, lv[0], lv[1])
            t12 = ht.Broot @ m34
            fld = np.einsum("ia,jb,abp,p->ij", ht.U[0], ht.U[1], ht.B12, t12).reshape(-1)
        total = coef * fld if total is None else total + coef * fld
    return total


def correction_moment(corr: Correction, g: PhaseGrid, psi) -> np.ndarray:
    """Moment of the separable correction: sum_terms dC_k(x) prod_mu sum_j vec_mu v^p Delta v."""
    total = np.zeros(corr.dC.shape[1])
    for coef, expo in psi:
        for k, vecs in corr.terms:
            s = 1.0
            for m, vec in enumerate(vecs):
                mu = g.dx + m
                s *= float(np.sum(vec * g.centres(mu) ** expo[m]) * g.h(mu))
            total = total + coef * s * corr.dC[k]
    return total


def moments(ht: HT, g: PhaseGrid) -> np.ndarray:
    """All moments of a state (HT + optional correction): array (n_mom, prod N_x)."""
    out = []
    for psi in moment_monomials(g.dv):
        fld = ht_moment(ht, g, psi)
        if ht.corr is not None:
            fld = fld + correction_moment(ht.corr, g, psi)
        out.append(fld)
    return np.stack(out)


def dense_moments(F: np.ndarray, g: PhaseGrid) -> np.ndarray:
    """Brute-force moments of a dense tensor by the midpoint sums of the definition."""
    vs = np.meshgrid(*[g.centres(g.dx + m) for m in range(g.dv)], indexing="ij")
    wv = float(np.prod([g.h(g.dx + m) for m in range(g.dv)]))
    Fm = F.reshape(int(np.prod(g.Nx)), -1)
    out = []
    for psi in moment_monomials(g.dv):
        w = np.zeros(vs[0].shape)
        for coef, expo in psi:
            t = np.full(vs[0].shape, coef)
            for m in range(g.dv):
                t = t * vs[m] ** expo[m]
            w = w + t
        out.append(Fm @ (w.reshape(-1) * wv))
    return np.stack(out)


# ----------------------------------------------------------------------------------------
# spectral operators and Poisson
# ----------------------------------------------------------------------------------------

def wavenumbers(g: PhaseGrid):
    """Per spatial dimension the derivative wavenumbers 2 pi m / L (Nyquist set to 0)."""
    ks = []
    for m in range(g.dx):
        n = g.N[m]
        L = g.hi[m] - g.lo[m]
        k = np.fft.fftfreq(n, d=1.0 / n) * (2.0 * np.pi / L)
        if n % 2 == 0:
            k[n // 2] = 0.0
        ks.append(k)
    return np.meshgrid(*ks, indexing="ij")


def deriv(f: np.ndarray, g: PhaseGrid, m: int) -> np.ndarray:
    """Spectral partial derivative d/dx_m of a flattened spatial field."""
    K = wavenumbers(g)
    fh = np.fft.fftn(f.reshape(g.Nx))
    return np.real(np.fft.ifftn(1j * K[m] * fh)).reshape(-1)


def div(vec: np.ndarray, g: PhaseGrid) -> np.ndarray:
    """Spectral divergence of a vector field (dx, prod N_x)."""
    return sum(deriv(vec[m], g, m) for m in range(g.dx))


def solve_poisson(s: np.ndarray, g: PhaseGrid) -> np.ndarray:
    """phi with -Lap(phi) = s, spectrally (modes with zero symbol get phi = 0)."""
    K = wavenumbers(g)
    K2 = sum(k * k for k in K)
    sh = np.fft.fftn(s.reshape(g.Nx))
    ph = np.where(K2 > 0.0, sh / np.where(K2 > 0.0, K2, 1.0), 0.0)
    return np.real(np.fft.ifftn(ph)).reshape(-1)


def poisson_field(rho: np.ndarray, g: PhaseGrid):
    """phi, E = -grad(phi) and the electric energy W = 1/2 sum |E|^2 Delta x^dx
    (Eq. Poisson, Eq. Efromphi, e_p = |E|^2/2 of Sec. 2.2)."""
    phi = solve_poisson(rho, g)
    E = np.stack([-deriv(phi, g, m) for m in range(g.dx)])
    cell = float(np.prod([g.h(m) for m in range(g.dx)]))
    W = 0.5 * float(np.sum(E * E)) * cell
    return phi, E, W


def field_energy_density(E: np.ndarray) -> np.ndarray:
    """e_p = |E|^2 / 2 pointwise."""
    return 0.5 * np.sum(E * E, axis=0)
