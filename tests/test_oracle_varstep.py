"""Pins of the oracle's variable-step BDF3 (Sec. 3.2.3: the classical variable-step BDF3 of
Gear with a step-ratio condition for stability) and of its adaptive step-size rule.

* Equal steps give the fixed-step Gear table (18/11, -9/11, 2/11; 6/11).
* The formula is exact on cubic polynomials for arbitrary step sequences and not on quartics
  (order exactly 3), which fixes every coefficient.
* On the Dahlquist problem y' = lam y with a non-uniform step pattern the error falls by 8
  when every step is halved.
* Zero stability: with a constant step ratio the two parasitic roots of the recurrence stay
  inside the unit disk at the ratio bound 1.4877 and leave it at 1.8.
* A variable-step oracle run conserves mass, momentum and energy to the Newton tolerance,
  and an equal-step sequence reproduces the fixed-step run bit for bit.
"""
import math

import numpy as np
import pytest

from oracle import macro, sl, stepper
from paper_2606_29027_b300 import inputs


def test_equal_steps_give_gear_table():
    for h in (0.1, 0.37, 2.0):
        a, beta = macro.bdf3_variable((h, h, h))
        assert np.allclose(a, (18 / 11, -9 / 11, 2 / 11), rtol=0, atol=1e-14)
        assert abs(beta - 6 / 11) < 1e-15


@pytest.mark.parametrize("seed", range(5))
def test_exact_on_cubics_not_on_quartics(seed):
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.05, 0.5, 3)
    t1 = rng.uniform(-1, 1)
    ts = [t1, t1 - h[0], t1 - h[0] - h[1], t1 - h[0] - h[1] - h[2]]
    a, beta = macro.bdf3_variable(h)
    c = rng.standard_normal(5)
    for deg in (0, 1, 2, 3):
        p = np.polynomial.Polynomial(c[: deg + 1])
        lhs = p(ts[0]) - beta * h[0] * p.deriv()(ts[0])
        rhs = a[0] * p(ts[1]) + a[1] * p(ts[2]) + a[2] * p(ts[3])
        assert abs(lhs - rhs) < 1e-12 * max(1.0, np.max(np.abs(c)))
    q = np.polynomial.Polynomial([0, 0, 0, 0, 1.0])
    lhs = q(ts[0]) - beta * h[0] * q.deriv()(ts[0])
    rhs = a[0] * q(ts[1]) + a[1] * q(ts[2]) + a[2] * q(ts[3])
    assert abs(lhs - rhs) > 1e-8


def _varstep_dahlquist(lam, T, n):
    """n steps over [0, T] in a repeating pattern of relative sizes (1, 1.3, 0.8, 1.1); the
    first three values exact (start-up)."""
    pat = np.array([1.0, 1.3, 0.8, 1.1])
    w = np.resize(pat, n)
    hs = T * w / w.sum()
    ts = np.concatenate([[0.0], np.cumsum(hs)])
    ys = [np.exp(lam * ts[k]) for k in range(3)]
    for k in range(3, n + 1):
        a, beta = macro.bdf3_variable((hs[k - 1], hs[k - 2], hs[k - 3]))
        rhs = a[0] * ys[-1] + a[1] * ys[-2] + a[2] * ys[-3]
        ys.append(rhs / (1 - beta * hs[k - 1] * lam))
    return ys[-1]


def test_third_order_with_variable_steps():
    lam, T = -1.3 + 0.7j, 2.0
    exact = np.exp(lam * T)
    errs = [abs(_varstep_dahlquist(lam, T, n) - exact) for n in (40, 80, 160)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 3.0) < 0.25), rates


@pytest.mark.parametrize("r,stable", [(1.0, True), (1.3, True), (macro.BDF3_RATIO_MAX, True),
                                      (1.8, False), (2.2, False)])
def test_zero_stability_at_constant_ratio(r, stable):
    a, _ = macro.bdf3_variable((r * r, r, 1.0))
    roots = np.roots([1.0, -a[0], -a[1], -a[2]])
    one = np.argmin(np.abs(roots - 1.0))
    assert abs(roots[one] - 1.0) < 1e-12        # consistency: the root 1
    parasitic = np.delete(np.abs(roots), one)
    assert (np.max(parasitic) < 1.0) == stable


def _run(w, dts):
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)
    Ws = [stepper.sl_step(st, dt, g, prm).W for dt in dts]
    return st, g, np.array(Ws)


def test_equal_variable_steps_reproduce_fixed_steps(monkeypatch):
    """Equal steps through the variable-step coefficients reproduce a run with the
    fixed-step Gear table substituted, to rounding."""
    w = inputs.landau_1d1v(N=(32, 64), alpha=0.2)
    _, _, W1 = _run(w, [0.1] * 6)
    monkeypatch.setattr(macro, "bdf3_variable", lambda h: (macro.BDF3["a"], macro.BDF3["beta"]))
    _, _, W2 = _run(w, [0.1] * 6)
    assert np.max(np.abs(W1 - W2) / np.abs(W2)) < 1e-11


def test_variable_step_run_conserves():
    w = inputs.landau_1d1v(N=(32, 64), alpha=0.3)
    dts = [0.1, 0.1, 0.12, 0.15, 0.1, 0.08, 0.11]
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)
    tot0 = stepper.totals(st, g)
    for dt in dts:
        assert stepper.sl_step(st, dt, g, prm).converged
    tot1 = stepper.totals(st, g)
    assert abs(tot1[0] - tot0[0]) <= 1e-12 * tot0[0]
    assert abs(tot1[1] - tot0[1]) <= 1e-12 * tot0[0]
    assert abs(tot1[2] - tot0[2]) <= 1e-12 * tot0[2]
    assert abs(st.t - sum(dts)) < 1e-14


def test_cfl_rule():
    """dt = cfl / max_i(a_i / Delta_i), capped by dt_max and by the ratio bound after the
    start-up; zero field: the x-advection by max|v| decides."""
    w = inputs.landau_1d1v(N=(32, 64), alpha=0.2)
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)
    vmax = float(np.max(np.abs(g.centres(1))))
    E = stepper.field_of(st.F, g, st.n_i)
    rate = max(vmax / g.h(0), float(np.max(np.abs(E))) / g.h(1))
    assert rate == vmax / g.h(0)
    assert abs(stepper.cfl_dt(st, g, 5.0, 10.0) - 5.0 / rate) < 1e-15
    assert stepper.cfl_dt(st, g, 5.0, 0.01) == 0.01
    for _ in range(3):
        stepper.sl_step(st, 0.05, g, prm)
    assert stepper.cfl_dt(st, g, 50.0, 10.0) == pytest.approx(macro.BDF3_RATIO_MAX * 0.05, rel=1e-15)
