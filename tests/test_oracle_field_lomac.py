"""Oracle pins: moments, spectral Poisson, and the adaptive-weight LoMaC projection
(Sec. 2; Sec. 3.2.1-3.2.2; Supp. B)."""
import math

import numpy as np
import pytest

from oracle import field, lomac, sl
from oracle import ht as htmod
from paper_2606_29027_b300 import inputs


def _grid(N, vmax=6.0, L=4 * math.pi):
    d = len(N)
    dx = d // 2
    return sl.PhaseGrid(dx, d - dx, N, (0.0,) * dx + (-vmax,) * dx, (L,) * dx + (vmax,) * dx)


@pytest.mark.parametrize("N,ranks", [((8, 16), (4, 5)), ((6, 5, 8, 7), (4, 3, 5, 4, 5, 6))])
@pytest.mark.parametrize("with_corr", [False, True])
def test_ht_moments_equal_dense_sums(N, ranks, with_corr):
    g = _grid(N)
    h = htmod.from_raw(inputs.random_ht(N, ranks, 2, smooth=False))
    if with_corr:
        rng = np.random.default_rng(0)
        dx = g.dx
        dC = rng.standard_normal((g.dv + 2, int(np.prod(N[:dx]))))
        terms = [(k, [rng.standard_normal(N[dx + m]) for m in range(g.dv)]) for k in range(g.dv + 2)]
        h.corr = htmod.Correction(dC=dC, terms=terms)
    got = field.moments(h, g)
    want = field.dense_moments(htmod.densify(h), g)
    assert got.shape[0] == field.n_moments(g.dv)
    assert np.allclose(got, want, atol=1e-12 * np.abs(want).max())


def test_maxwellian_moments():
    """Landau f0 on [-6,6]: M0 = 1 + alpha cos(kx), M1 = 0, M2 = M0, <v^3 f> = 0 up to the
    truncated Maxwellian tails and the midpoint rule."""
    w = inputs.landau_1d1v(N=(32, 128), alpha=0.3)
    g = sl.PhaseGrid(1, 1, w.N, w.lo, w.hi)
    F = htmod.from_terms(inputs.initial_factors(w))
    mom = field.moments(F, g)
    x = g.centres(0)
    assert np.allclose(mom[0], 1 + 0.3 * np.cos(0.5 * x), atol=1e-8)
    assert np.allclose(mom[1], 0.0, atol=1e-14)
    assert np.allclose(mom[2], 1 + 0.3 * np.cos(0.5 * x), atol=1e-6)
    assert np.allclose(mom[4], 0.0, atol=1e-13)


def test_poisson_landau_closed_form():
    """rho = -alpha cos(kx): E = -(alpha/k) sin(kx), W = alpha^2 L / (4 k^2) (Sec. 4.1 Landau)."""
    alpha, k = 0.01, 0.5
    L = 2 * math.pi / k
    g = sl.PhaseGrid(1, 1, (64, 8), (0, -1), (L, 1))
    x = g.centres(0)
    phi, E, W = field.poisson_field(-alpha * np.cos(k * x), g)
    assert np.allclose(E[0], -(alpha / k) * np.sin(k * x), atol=1e-15)
    assert np.allclose(phi, -(alpha / k ** 2) * np.cos(k * x), atol=1e-15)
    assert W == pytest.approx(alpha ** 2 * L / (4 * k ** 2), rel=1e-12)
    assert W == pytest.approx(4 * math.pi * 1e-4, rel=1e-12)


def test_poisson_2d_two_modes():
    alpha, k = 0.01, 0.5
    L = 2 * math.pi / k
    g = sl.PhaseGrid(2, 2, (32, 32, 4, 4), (0, 0, -1, -1), (L, L, 1, 1))
    X, Y = np.meshgrid(g.centres(0), g.centres(1), indexing="ij")
    rho = -alpha * (np.cos(k * X) + np.cos(k * Y))
    _, E, W = field.poisson_field(rho.reshape(-1), g)
    assert W == pytest.approx(alpha ** 2 * L * L / (2 * k ** 2), rel=1e-12)
    assert np.allclose(E[0].reshape(32, 32), -(alpha / k) * np.sin(k * X), atol=1e-15)


def test_poisson_against_direct_dft():
    """-Lap(phi) = rho checked with an O(N^2) direct DFT written out here, on a random field
    (independent of numpy's FFT)."""
    rng = np.random.default_rng(1)
    N, L = 12, 3.0
    g = sl.PhaseGrid(1, 1, (N, 4), (0, -1), (L, 1))
    rho = rng.standard_normal(N)
    rho -= rho.mean()
    phi = field.solve_poisson(rho, g)
    j = np.arange(N)
    m = np.where(j <= N // 2, j, j - N)
    F = np.exp(-2j * math.pi * np.outer(m, j) / N)
    kk = 2 * math.pi * m / L
    kk[N // 2] = 0.0
    rho_h = F @ rho
    phi_h = F @ phi
    mask = kk != 0
    assert np.allclose(kk[mask] ** 2 * phi_h[mask], rho_h[mask], atol=1e-12)
    assert abs(phi_h[0]) < 1e-12 and abs(phi_h[N // 2]) < 1e-12


def test_spectral_identities():
    """div(grad f) = -|k|^2 f (compatible operators) and sum_x rho E = 0 (momentum source has
    zero total), Sec. 3.2.3."""
    rng = np.random.default_rng(4)
    g = sl.PhaseGrid(2, 2, (16, 12, 2, 2), (0, 0, -1, -1), (3.0, 5.0, 1, 1))
    f = rng.standard_normal(16 * 12)
    f -= f.mean()
    lap = field.div(np.stack([field.deriv(f, g, 0), field.deriv(f, g, 1)]), g)
    _, E, _ = field.poisson_field(f, g)
    assert abs(float(np.sum(f * E[0]))) < 1e-12 and abs(float(np.sum(f * E[1]))) < 1e-12
    # -lap(phi) reproduces rho on the resolvable modes: apply twice and compare
    u = field.solve_poisson(f, g)
    lap_u = field.div(np.stack([field.deriv(u, g, 0), field.deriv(u, g, 1)]), g)
    f2 = field.solve_poisson(-lap_u, g)
    assert np.allclose(f2, u, atol=1e-12)


# ----------------------------------------------------------------------------------------
# LoMaC (Supp. B)
# ----------------------------------------------------------------------------------------

def _basis(dv, Nv, seed, vmax=6.0):
    rng = np.random.default_rng(seed)
    B = []
    for m in range(dv):
        v = -vmax + (np.arange(Nv) + 0.5) * (2 * vmax / Nv)
        om = np.exp(-(v - 0.3 * m) ** 2 / 2) * (1 + 0.2 * rng.random(Nv)) + 1e-12
        B.append(lomac.gram_schmidt_1d(om, v, 2 * vmax / Nv))
    return B


@pytest.mark.parametrize("dv", [1, 2])
def test_q_basis_orthogonal_and_norms(dv):
    """Q0, Q1_mu, Q2 are mutually orthogonal under <.,.>_{v;omega^{-1}} and their squared norms
    equal the tensor-product formulas (Supp. B.2)."""
    Nv = 20
    B = _basis(dv, Nv, 3)
    terms = lomac.velocity_terms(B)
    Q = []
    for k in range(dv + 2):
        t = 0
        for kk, vecs in terms:
            if kk != k:
                continue
            p = vecs[0]
            for vec in vecs[1:]:
                p = np.multiply.outer(p, vec)
            t = t + p
        Q.append(t)
    Om = B[0].omega
    for b in B[1:]:
        Om = np.multiply.outer(Om, b.omega)
    wv = np.prod([b.wq for b in B])
    ip = lambda a, b: float(np.sum(a * b * wv / Om))
    n0, n1, n2 = lomac.q_norms(B)
    norms = [n0] + n1 + [n2]
    for a in range(dv + 2):
        for b in range(dv + 2):
            val = ip(Q[a], Q[b])
            if a == b:
                assert val == pytest.approx(norms[a], rel=1e-12)
            else:
                assert abs(val) <= 1e-12 * math.sqrt(norms[a] * norms[b])


@pytest.mark.parametrize("dv", [1, 2])
def test_projection_closed_form_equals_weighted_least_squares(dv):
    """P* F from the closed-form coefficients (Eq. C0_def..C2_def) equals the weighted
    least-squares projection solved by dense normal equations; it is idempotent and it
    preserves M0, M1, M2 (Eq. moments_pres_disc)."""
    Nx, Nv = 5, 14
    N = (Nx,) * dv + (Nv,) * dv
    g = sl.PhaseGrid(dv, dv, N, (0.0,) * dv + (-6.0,) * dv, (1.0,) * dv + (6.0,) * dv)
    B = _basis(dv, Nv, 7)
    F = np.random.default_rng(2).standard_normal(N)
    P = lomac.project_dense(F, B, g)
    assert np.allclose(P, lomac.weighted_lsq_projection(F, B, g), atol=1e-11 * np.abs(P).max())
    assert np.allclose(lomac.project_dense(P, B, g), P, atol=1e-11 * np.abs(P).max())
    mF = field.dense_moments(F, g)[: dv + 2]
    mP = field.dense_moments(P, g)[: dv + 2]
    assert np.allclose(mP, mF, atol=1e-11 * np.abs(mF).max())


def test_weight_floor_positive():
    u = np.array([0.5, -0.3, 1e-20, 0.0, -1e-15])
    om = lomac.weight_from_leaf(u, 1e-12)
    assert np.all(om >= 1e-12) and om[1] == 0.3


@pytest.mark.parametrize("N", [(8, 16), (6, 6, 10, 10)])
def test_lomac_update_matches_target_moments(N):
    """U(F^{n+1}) = U^{n+1} for F^{n+1} = F* - R(U(F*)) + R(U^{n+1}) (Eq. LoMaC_update_discrete),
    with R(U(F*)) = P* F* checked densely (Supp. B.3)."""
    g = _grid(N)
    w = inputs.landau_1d1v(N=N, alpha=0.2) if len(N) == 2 else inputs.landau_2d2v(n=N[0], alpha=0.2)
    w.N, w.lo, w.hi = N, g.lo, g.hi
    Fs = htmod.truncate(htmod.from_terms(inputs.initial_factors(w)), 1e-13, 10)
    # perturb so that F* is not exactly in the projection range
    raw = inputs.random_ht(N, [3] * len(N) + ([3, 3] if len(N) == 4 else []), 5, smooth=True)
    pert = htmod.from_raw(raw)
    Fs = htmod.truncate(htmod.HT(U=[np.hstack([a, 1e-3 * b]) for a, b in zip(Fs.U, pert.U)],
                                 Broot=_blockdiag(Fs.Broot, pert.Broot),
                                 B12=None if len(N) == 2 else _blockdiag3(Fs.B12, pert.B12),
                                 B34=None if len(N) == 2 else _blockdiag3(Fs.B34, pert.B34)), 1e-13, 30)
    n_i = float(np.mean(field.moments(Fs, g)[0]))
    B = lomac.basis_from_ht(Fs, g)
    U_star = lomac.conserved_from_moments(field.moments(Fs, g), g, n_i)
    # R(U(F*)) equals P* F*
    C_from_U = lomac.coefficients_from_U(U_star, B, g, n_i)
    P_dense = lomac.project_dense(htmod.densify(Fs), B, g)
    assert np.allclose(lomac.expand_dense(C_from_U, lomac.velocity_terms(B), g), P_dense,
                       atol=1e-11 * np.abs(P_dense).max())
    U_t = U_star * (1 + 0.01 * np.random.default_rng(0).standard_normal(U_star.shape))
    Fn = lomac.correct(Fs, B, U_t, g, n_i)
    U_new = lomac.conserved_from_moments(field.moments(Fn, g), g, n_i)
    assert np.allclose(U_new, U_t, rtol=0, atol=1e-13 * np.abs(U_t).max())


def _blockdiag(A, B):
    out = np.zeros((A.shape[0] + B.shape[0], A.shape[1] + B.shape[1]))
    out[: A.shape[0], : A.shape[1]] = A
    out[A.shape[0]:, A.shape[1]:] = B
    return out


def _blockdiag3(A, B):
    out = np.zeros(tuple(a + b for a, b in zip(A.shape, B.shape)))
    out[: A.shape[0], : A.shape[1], : A.shape[2]] = A
    out[A.shape[0]:, A.shape[1]:, A.shape[2]:] = B
    return out
