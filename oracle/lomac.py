"""Adaptive-weight LoMaC projection: discrete weight, 1D weighted Gram-Schmidt, the
orthogonal basis Q, closed-form coefficients C, the reconstruction R(U) and the update
(Sec. 3.2.1-3.2.2, Eq. LoMaC_update_discrete; Supp. B.1-B.3).

Test infrastructure: part of the FP64 oracle, never called by the CUDA path.

Readings: the floor delta is not given by the paper; delta = 1e-12 is applied to the
Euclidean-unit leading leaf column (Supp. B.1 only asks for a small delta independent of
mu).  The weight is built from the velocity leaves of F* after HSVD truncation and kept
fixed through the Newton solve.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np

from . import field
from .ht import HT, Correction
from .sl import PhaseGrid

DELTA_DEFAULT = 1e-12


@dataclass
class Basis1D:
    v: np.ndarray        # grid v^(mu)
    wq: float            # quadrature weight Delta v^(mu)
    omega: np.ndarray    # omega^(mu),*
    q1: np.ndarray
    q2: np.ndarray
    gamma: float
    eta: float
    beta: float
    n0: float            # ||omega||^2
    n1: float            # ||q1||^2
    n2: float            # ||q2||^2


def inner_1d(p, q, omega, wq):
    """<p, q>_{v^(mu); omega^{-1}} = sum p q w / omega (Supp. B.1)."""
    return float(np.sum(p * q * wq / omega))


def weight_from_leaf(u1: np.ndarray, delta: float) -> np.ndarray:
    """omega^(mu),* = max(|u_1^(mu)|, delta) elementwise (Supp. B.1, Eq. omega_star_tensor
    and the positivity floor)."""
    return np.maximum(np.abs(u1), delta)


def gram_schmidt_1d(omega: np.ndarray, v: np.ndarray, wq: float) -> Basis1D:
    """Weighted Gram-Schmidt of {omega, v omega, v^2 omega} (Supp. B.2)."""
    vw = v * omega
    v2w = v * v * omega
    n0 = inner_1d(omega, omega, omega, wq)
    gamma = inner_1d(vw, omega, omega, wq) / n0
    q1 = vw - gamma * omega
    eta = inner_1d(v2w, omega, omega, wq) / n0
    n1 = inner_1d(q1, q1, omega, wq)
    beta = inner_1d(v2w, q1, omega, wq) / n1
    q2 = v2w - eta * omega - beta * q1
    n2 = inner_1d(q2, q2, omega, wq)
    return Basis1D(v=v, wq=wq, omega=omega, q1=q1, q2=q2, gamma=gamma, eta=eta, beta=beta,
                   n0=n0, n1=n1, n2=n2)


def basis_from_ht(ht: HT, g: PhaseGrid, delta: float = DELTA_DEFAULT) -> List[Basis1D]:
    """Per velocity dimension: weight from column 0 of the (truncated) velocity leaf basis,
    then the 1D Gram-Schmidt (Supp. B.1-B.2)."""
    out = []
    for m in range(g.dv):
        mu = g.dx + m
        om = weight_from_leaf(ht.U[mu][:, 0], delta)
        out.append(gram_schmidt_1d(om, g.centres(mu), g.h(mu)))
    return out


def q_norms(B: List[Basis1D]):
    """||Q0||^2, ||Q1_mu||^2 (list), ||Q2||^2 by the tensor-product formulas (Supp. B.2)."""
    dv = len(B)
    p0 = float(np.prod([b.n0 for b in B]))
    n1 = [B[m].n1 * float(np.prod([B[o].n0 for o in range(dv) if o != m])) for m in range(dv)]
    n2 = sum(B[m].n2 * float(np.prod([B[o].n0 for o in range(dv) if o != m])) for m in range(dv))
    return p0, n1, n2


def coefficients(M0, M1, M2, B: List[Basis1D]):
    """C0, C1_mu, C2 from raw moments (Eq. C0_def, C1_def, C2_def).  Returns (dv+2, Nx)."""
    dv = len(B)
    nQ0, nQ1, nQ2 = q_norms(B)
    C0 = M0 / nQ0
    C1 = [(M1[m] - B[m].gamma * M0) / nQ1[m] for m in range(dv)]
    num2 = M2 - sum(b.eta for b in B) * M0
    for m in range(dv):
        num2 = num2 - B[m].beta * (M1[m] - B[m].gamma * M0)
    C2 = num2 / nQ2
    return np.stack([C0] + C1 + [C2])


def velocity_terms(B: List[Basis1D]):
    """Separable pieces of Q0, Q1_mu, Q2 as (k, [vec_mu]) (Supp. B.2):
    Q0 = (x)omega; Q1_mu = omega..q1^(mu)..omega; Q2 = sum_mu omega..q2^(mu)..omega."""
    dv = len(B)
    terms = [(0, [b.omega for b in B])]
    for m in range(dv):
        terms.append((1 + m, [B[o].q1 if o == m else B[o].omega for o in range(dv)]))
    for m in range(dv):
        terms.append((1 + dv, [B[o].q2 if o == m else B[o].omega for o in range(dv)]))
    return terms


def raw_from_conserved(U: np.ndarray, g: PhaseGrid, n_i: float):
    """M0 = U0, M1 = U1, M2 = 2 (U2 - e_p(U0)) with m_e = 1 (Eq. M from U); e_p from the
    spectral Poisson solve of rho = n_i - U0 (Eq. charge_density)."""
    dv = g.dv
    _, E, _ = field.poisson_field(n_i - U[0], g)
    ep = field.field_energy_density(E)
    return U[0], [U[1 + m] for m in range(dv)], 2.0 * (U[1 + dv] - ep)


def conserved_from_moments(mom: np.ndarray, g: PhaseGrid, n_i: float) -> np.ndarray:
    """U = (M0, M1, M2/2 + e_p(M0)) (Eq. macro_sys_comp with m_e = 1)."""
    dv = g.dv
    _, E, _ = field.poisson_field(n_i - mom[0], g)
    ep = field.field_energy_density(E)
    return np.stack([mom[0]] + [mom[1 + m] for m in range(dv)] + [0.5 * mom[1 + dv] + ep])


def coefficients_from_U(U, B, g, n_i):
    """C-tilde(U): the coefficients of R(U) (Supp. B.3, Eq. reconstruction_supp)."""
    M0, M1, M2 = raw_from_conserved(U, g, n_i)
    return coefficients(M0, M1, M2, B)


def coefficients_from_moments(mom, B, g):
    dv = g.dv
    return coefficients(mom[0], [mom[1 + m] for m in range(dv)], mom[1 + dv], B)


def correct(Fstar: HT, B: List[Basis1D], U_target: np.ndarray, g: PhaseGrid, n_i: float) -> HT:
    """F^{n+1} = F* - R(U(F*)) + R(U^{n+1}) (Eq. LoMaC_update_discrete), kept exactly as the
    HT of F* plus the separable term sum_k (C~_k(U^{n+1}) - C_k(F*)) (x) Q_k."""
    mom = field.moments(Fstar, g)
    dC = coefficients_from_U(U_target, B, g, n_i) - coefficients_from_moments(mom, B, g)
    if Fstar.corr is not None:
        raise ValueError("F* must be a plain HT (the output of SLAR)")
    out = Fstar.without_correction()
    out.corr = Correction(dC=dC, terms=velocity_terms(B))
    return out


def project_dense(F: np.ndarray, B: List[Basis1D], g: PhaseGrid) -> np.ndarray:
    """P* F for a dense tensor: coefficients from its raw moments, then sum C_k (x) Q_k
    (Eq. phase_proj_closed)."""
    mom = field.dense_moments(F, g)
    C = coefficients_from_moments(mom, B, g)
    return expand_dense(C, velocity_terms(B), g)


def expand_dense(C: np.ndarray, terms, g: PhaseGrid) -> np.ndarray:
    Nv = g.N[g.dx:]
    out = np.zeros((C.shape[1],) + Nv)
    for k, vecs in terms:
        t = vecs[0]
        for vec in vecs[1:]:
            t = np.multiply.outer(t, vec)
        out = out + np.multiply.outer(C[k], t)
    return out.reshape(g.N)


def weighted_lsq_projection(F: np.ndarray, B: List[Basis1D], g: PhaseGrid) -> np.ndarray:
    """Brute force P*: per spatial point solve the weighted normal equations for the span of
    {Omega, V_mu Omega, |V|^2 Omega} under <G, H> = sum G H w^v / Omega (Supp. B.1,
    Eq. inner_velocity).  Independent of the Gram-Schmidt closed form."""
    Nv = g.N[g.dx:]
    vs = np.meshgrid(*[b.v for b in B], indexing="ij")
    Om = B[0].omega
    for b in B[1:]:
        Om = np.multiply.outer(Om, b.omega)
    wv = float(np.prod([b.wq for b in B]))
    funcs = [Om] + [vs[m] * Om for m in range(g.dv)] + [sum(vs[m] ** 2 for m in range(g.dv)) * Om]
    Phi = np.stack([f.reshape(-1) for f in funcs], axis=1)          # (Nv, dv+2)
    W = (wv / Om).reshape(-1)
    Gm = Phi.T @ (W[:, None] * Phi)
    Fm = F.reshape(-1, Phi.shape[0])
    rhs = (Fm * W[None, :]) @ Phi
    coef = np.linalg.solve(Gm, rhs.T).T
    return (coef @ Phi.T).reshape(g.N)


def flux_tables(B: List[Basis1D], g: PhaseGrid):
    """<psi Q_k>_v for every moment weight psi and basis function Q_k: (n_mom, dv+2)."""
    terms = velocity_terms(B)
    mons = field.moment_monomials(g.dv)
    T = np.zeros((len(mons), g.dv + 2))
    for a, psi in enumerate(mons):
        for coef, expo in psi:
            for k, vecs in terms:
                s = 1.0
                for m, vec in enumerate(vecs):
                    s *= float(np.sum(vec * B[m].v ** expo[m]) * B[m].wq)
                T[a, k] += coef * s
    return T
