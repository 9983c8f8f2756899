"""Linear dispersion relations used as physics pins of the Vlasov-Poisson oracle.

Test infrastructure: part of the FP64 oracle, never called by the CUDA path.

For a sum of drifting Maxwellians with densities n_s, drifts u_s and temperatures T_s
(velocity variances; 1 unless given), the electrostatic dielectric function (electron
charge -1, omega_p = 1 for total density 1, rescaling of Sec. 2.1) is

    eps(k, w) = 1 + sum_s (n_s / T_s) (1 + zeta_s Z(zeta_s)) / k^2,
    zeta_s = (w - k u_s) / (k sqrt(2 T_s)),

with the plasma dispersion function Z(z) = i sqrt(pi) w(z) (Faddeeva function).  A zero
of eps gives the complex frequency; Im w is the amplitude growth (damping) rate of E.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import wofz


def plasma_Z(z: complex) -> complex:
    return 1j * math.sqrt(math.pi) * complex(wofz(z))


def dielectric(k: float, w: complex, species) -> complex:
    """species: tuples (n_s, u_s) or (n_s, u_s, T_s)."""
    out = 1.0 + 0j
    for sp in species:
        n_s, u_s = sp[0], sp[1]
        T_s = sp[2] if len(sp) > 2 else 1.0
        z = (w - k * u_s) / (k * math.sqrt(2.0 * T_s))
        out += (n_s / T_s) * (1.0 + z * plasma_Z(z)) / (k * k)
    return out


def root(k: float, w0: complex, species=((1.0, 0.0),), iters: int = 100) -> complex:
    """Secant iteration for eps(k, w) = 0 from the initial guess w0."""
    w_prev, w = w0, w0 * (1.0 + 1e-3) + 1e-3j
    f_prev, f = dielectric(k, w_prev, species), dielectric(k, w, species)
    for _ in range(iters):
        if f == f_prev:
            break
        w_new = w - f * (w - w_prev) / (f - f_prev)
        w_prev, f_prev = w, f
        w, f = w_new, dielectric(k, w_new, species)
        if abs(w - w_prev) < 1e-14:
            break
    return w


def landau_rate(k: float = 0.5) -> complex:
    """Least-damped Langmuir root of a unit Maxwellian."""
    return root(k, 1.4 - 0.15j)


def two_stream_rate(k: float, v0: float, n_beam: float = 0.5) -> complex:
    """Unstable root of two beams of density n_beam each at +-v0 (0.5: total density 1, as in
    the 2D-2V workload; 1.0: the 1D-1V example of Sec. 4.1, whose two unit Gaussians have
    total density 2)."""
    return root(k, 0.0 + 0.3j, species=((n_beam, v0), (n_beam, -v0)))


def bump_on_tail_rate(k: float = 0.3, u: float = 4.5, vt: float = 0.5) -> complex:
    """Unstable root of the 1D-1V bump-on-tail data of Sec. 4.1: a unit-temperature bulk of
    density 0.9 (n_p exp(-v^2/2), n_p = 9/(10 sqrt(2 pi))) and a beam of temperature vt at u
    of density 0.2 sqrt(vt) (n_b exp(-(v - u)^2/(2 vt)), n_b = 2/(10 sqrt(2 pi)))."""
    return root(k, 1.0 + 0.1j, species=((0.9, 0.0, 1.0), (0.2 * math.sqrt(vt), u, vt)))
