"""Oracle pins: time integrators and the JFNK macroscopic solve (Sec. 3.2.3; Sec. 4)."""
import math

import numpy as np
import pytest

from oracle import field, lomac, macro, sl, stepper
from oracle import ht as htmod
from paper_2606_29027_b300 import inputs


def test_dirk3_gamma_and_order_conditions():
    """Alexander's S-stable DIRK3: gamma solves x^3 - 3x^2 + 3x/2 - 1/6 = 0; the tableau
    satisfies the order-3 conditions and is stiffly accurate."""
    A, c = macro.dirk3_tableau()
    g = macro.DIRK3_GAMMA
    assert abs(g ** 3 - 3 * g ** 2 + 1.5 * g - 1 / 6) < 1e-15
    b = A[2]
    assert np.allclose(A.sum(axis=1), c)
    assert b.sum() == pytest.approx(1.0, abs=1e-15)
    assert b @ c == pytest.approx(0.5, abs=1e-14)
    assert b @ c ** 2 == pytest.approx(1 / 3, abs=1e-14)
    assert b @ A @ c == pytest.approx(1 / 6, abs=1e-14)
    # S-stability: R(z) -> 0 as z -> -inf for a stiffly accurate L-stable method
    z = -1e8
    R = 1 + z * b @ np.linalg.solve(np.eye(3) - z * A, np.ones(3))
    assert abs(R) < 1e-6


def _dirk3_solve(lam, T, n):
    A, c = macro.dirk3_tableau()
    h = T / n
    y = 1.0
    for _ in range(n):
        K = []
        for i in range(3):
            rhs = y + h * sum(A[i, j] * K[j] for j in range(i))
            yi = rhs / (1 - h * A[i, i] * lam)
            K.append(lam * yi)
        y = yi
    return y


def _bdf3_solve(lam, T, n):
    h = T / n
    ys = [np.exp(lam * h * k) for k in range(3)]
    a, beta = macro.BDF3["a"], macro.BDF3["beta"]
    for k in range(3, n + 1):
        rhs = a[0] * ys[-1] + a[1] * ys[-2] + a[2] * ys[-3]
        ys.append(rhs / (1 - beta * h * lam))
    return ys[-1]


@pytest.mark.parametrize("solver", [_dirk3_solve, _bdf3_solve])
def test_third_order_on_dahlquist(solver):
    lam, T = -1.3 + 0.7j, 2.0
    exact = np.exp(lam * T)
    errs = [abs(solver(lam, T, n) - exact) for n in (20, 40, 80)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 3.0) < 0.25), rates


def _tiny_closure(N=(8, 16), seed=0):
    w = inputs.landau_1d1v(N=N, alpha=0.3)
    g = sl.PhaseGrid(1, 1, N, w.lo, w.hi)
    F0 = htmod.truncate(htmod.from_terms(inputs.initial_factors(w)), 1e-12, 8)
    n_i = float(np.mean(field.moments(F0, g)[0]))
    E = field.poisson_field(n_i - field.moments(F0, g)[0], g)[1]
    Fs = htmod.truncate(htmod.HT(U=F0.U, Broot=F0.Broot), 1e-12, 8)
    from oracle import cross
    Fs = cross.htaca(lambda idx: sl.sl_eval(F0, E, 0.5, idx, g), N, 1e-10, 16)
    cl = macro.make_closure(Fs, g, n_i)
    U0 = lomac.conserved_from_moments(field.moments(F0, g), g, n_i)
    return cl, U0, g


def test_jfnk_matches_dense_newton():
    """JFNK (GMRES, finite-difference J v) reaches the same root as a dense Newton method
    with a full finite-difference Jacobian on a tiny grid."""
    cl, U0, g = _tiny_closure()
    dt = 0.4
    Gfun = lambda U: U - U0 - dt * macro.K_operator(U, cl)
    Ustar = lomac.conserved_from_moments(cl.mom_star, g, cl.n_i)
    U_j, st = macro.jfnk(Gfun, Ustar, 1e-13, 1e-6)
    assert st.converged
    # dense Newton
    U = Ustar.copy()
    n = U.size
    for _ in range(12):
        G0 = Gfun(U).reshape(-1)
        if np.max(np.abs(G0)) < 1e-14:
            break
        J = np.zeros((n, n))
        h = 1e-7
        for c in range(n):
            e = np.zeros(n)
            e[c] = h
            J[:, c] = (Gfun((U.reshape(-1) + e).reshape(U.shape)).reshape(-1) - G0) / h
        U = U - np.linalg.solve(J, G0).reshape(U.shape)
    assert np.allclose(U_j, U, atol=1e-11)


def test_macro_residual_conserves_totals():
    """Sum over x of K(U) has zero mass and energy components (flux form) and zero momentum
    (spectral sum rho E = 0): the discrete totals change only through the Newton residual."""
    cl, U0, g = _tiny_closure()
    U = U0 * (1 + 0.01 * np.random.default_rng(3).standard_normal(U0.shape))
    K = macro.K_operator(U, cl)
    assert np.allclose(K.sum(axis=1), 0.0, atol=1e-12)


def test_gmres_solves_linear_system():
    rng = np.random.default_rng(0)
    A = np.eye(40) * 3 + 0.3 * rng.standard_normal((40, 40))
    b = rng.standard_normal(40)
    x, its = macro.gmres(lambda v: A @ v, b, 1e-12, 10, 400)
    assert np.linalg.norm(A @ x - b) <= 1e-11 * np.linalg.norm(b)
