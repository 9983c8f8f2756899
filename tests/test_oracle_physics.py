"""End-to-end physics pins of the oracle: linear Landau damping and conservation with the
LoMaC correction (Sec. 4.1 Landau damping; Sec. 3.2.2 U(F^{n+1}) = U^{n+1})."""
import math
import os

import numpy as np
import pytest

from oracle import dispersion, field, sl, stepper
from paper_2606_29027_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_root():
    vals = {}
    with open(os.path.join(GOLDEN, "landau_root.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()
                vals[k] = float(v)
    return vals


def test_dispersion_root_matches_golden():
    gr = _golden_root()
    w = dispersion.landau_rate(gr["k"])
    assert w.real == pytest.approx(gr["omega_re"], abs=2e-4)
    assert w.imag == pytest.approx(gr["omega_im"], abs=2e-4)


def test_two_stream_root_tends_to_the_cold_beam_root():
    """Fast, narrow beams (k v_t << |w - k v0|): the warm two-stream root approaches the
    closed-form root of two cold half-density beams, w^2 = ((2a^2 + 1) - sqrt(8a^2 + 1)) / 2
    with a = k v0 (purely growing for a < 1), and the thermal correction shrinks with k v_t at
    fixed a."""
    def cold(a):
        return math.sqrt(-((2 * a * a + 1) - math.sqrt(8 * a * a + 1)) / 2)

    errs = []
    for v0, k in ((20.0, 0.03), (40.0, 0.015)):
        w = dispersion.two_stream_rate(k, v0)
        assert abs(w.real) < 1e-10
        errs.append(abs(w.imag - cold(k * v0)) / cold(k * v0))
    assert errs[0] < 1e-2
    assert errs[1] < errs[0] / 2


@pytest.mark.parametrize("T", [0.25, 2.0])
@pytest.mark.parametrize("k", [0.4, 0.5])
def test_dispersion_temperature_scaling(T, k):
    """eps(k, w; n, T) = eps(k sqrt(T), w; n, 1): zeta = w / (k sqrt(2T)) and n / (T k^2)
    depend on k and T only through k sqrt(T), so the roots coincide."""
    r1 = dispersion.root(k, 1.4 - 0.15j, species=((1.0, 0.0, T),))
    r2 = dispersion.root(k * math.sqrt(T), 1.4 - 0.15j, species=((1.0, 0.0, 1.0),))
    assert abs(r1 - r2) < 1e-12


def _run_landau(steps, lomac=True, foot_flip=False, monkeypatch=None):
    w = inputs.landau_1d1v()
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap, lomac=lomac)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)
    tot0 = stepper.totals(st, g)
    ts, Ws = [0.0], [field.poisson_field(st.n_i - st.U[0], g)[2]]
    for _ in range(steps):
        s = stepper.sl_step(st, w.dt, g, prm)
        assert s.converged or not lomac
        ts.append(st.t)
        Ws.append(s.W)
    return np.array(ts), np.array(Ws), tot0, stepper.totals(st, g)


def _fit_rate(ts, Ws, t0=2.0, t1=20.0):
    A = np.sqrt(Ws)
    pk = [i for i in range(1, len(A) - 1) if A[i] > A[i - 1] and A[i] >= A[i + 1] and t0 <= ts[i] <= t1]
    return np.polyfit(ts[pk], np.log(A[pk]), 1)[0], len(pk)


@pytest.mark.slow
def test_weak_landau_damping_rate_and_conservation():
    """1D-1V weak Landau (alpha = 0.01, k = 0.5, 64 x 128, dt = 0.1, eps = 1e-6, cap 16):
    the amplitude of E decays at the linear rate (within 2%) and mass, momentum and energy
    are conserved to the Newton tolerance."""
    ts, Ws, tot0, tot1 = _run_landau(200)
    rate, npk = _fit_rate(ts, Ws)
    want = dispersion.landau_rate(0.5).imag
    assert npk >= 6
    assert abs(rate - want) <= _golden_root()["rel_tol_rate"] * abs(want), rate
    drift = np.abs(tot1 - tot0)
    assert drift[0] <= 1e-12 * abs(tot0[0])
    assert drift[-1] <= 1e-12 * abs(tot0[-1])
    assert drift[1] <= 1e-12 * abs(tot0[0])


@pytest.mark.slow
def test_two_stream_growth_rate_1d1v():
    """1D-1V two-stream instability with the initial data of the paper's example (Sec. 4.1:
    two unit-density Maxwellian beams at +-2.4, alpha = 1e-3, k = 0.2, x in [0, 10 pi),
    v in [-8, 8]; here 64 x 128, dt = 0.1, eps = 1e-5): in the linear phase the k = 0.2
    Fourier mode of E grows at the rate of the dispersion root of two unit-density beams
    (0.273).  The fit over t in [12, 24] still holds a few percent of beating with the damped
    modes, hence 6 %; half-density beams (0.226), a flipped force or a mis-scaled field are
    far outside."""
    w = inputs.two_stream_1d1v()
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)

    def mode1():
        E = np.asarray(field.poisson_field(st.n_i - st.U[0], g)[1]).reshape(-1)
        return abs(np.fft.fft(E)[1])

    ts, amp = [0.0], [mode1()]
    for _ in range(240):
        s = stepper.sl_step(st, w.dt, g, prm)
        assert s.converged
        ts.append(st.t)
        amp.append(mode1())
    ts, amp = np.array(ts), np.array(amp)
    m = (ts >= 12.0) & (ts <= 24.0)
    rate = np.polyfit(ts[m], np.log(amp[m]), 1)[0]
    want = dispersion.two_stream_rate(w.k, 2.4, n_beam=1.0).imag
    assert abs(rate - want) <= 0.06 * want, (rate, want)
    assert abs(rate - dispersion.two_stream_rate(w.k, 2.4).imag) > 0.1 * want


@pytest.mark.slow
def test_bump_on_tail_growth_rate_1d1v():
    """1D-1V bump-on-tail instability with the data of the paper's example (Sec. 4.1: bulk
    n_p exp(-v^2/2) and beam n_b exp(-(v - 4.5)^2 / (2 * 0.5)), k = 0.3, x in [0, 20 pi / 3),
    v in [-13, 13]; here 64 x 128, dt = 0.1, eps = 1e-6) at a perturbation of 1e-4 instead of
    the example's 0.04, which saturates before the beam-driven wave dominates the beating with
    the bulk Langmuir waves: the k = 0.3 Fourier mode of E grows at the rate of the unstable
    dispersion root of a bulk and a drifting beam of temperature 0.5 (0.192), within 3 % over
    t in [15, 40]."""
    w = inputs.bump_on_tail_1d1v(alpha=1e-4, eps=1e-6)
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)

    def mode1():
        E = np.asarray(field.poisson_field(st.n_i - st.U[0], g)[1]).reshape(-1)
        return abs(np.fft.fft(E)[1])

    ts, amp = [0.0], [mode1()]
    for _ in range(400):
        s = stepper.sl_step(st, w.dt, g, prm)
        assert s.converged
        ts.append(st.t)
        amp.append(mode1())
    ts, amp = np.array(ts), np.array(amp)
    m = (ts >= 15.0) & (ts <= 40.0)
    rate = np.polyfit(ts[m], np.log(amp[m]), 1)[0]
    want = dispersion.bump_on_tail_rate(w.k).imag
    assert abs(rate - want) <= 0.03 * want, (rate, want)


def test_wrong_force_sign_is_caught(monkeypatch):
    """A planted mistake in the oracle (foot velocity v - E tau instead of v + E tau) turns
    damping into growth; the Landau pin catches it."""
    orig = sl.trace_feet

    def flipped(idx, E, tau, g, foot="rk3"):
        return orig(idx, -E, tau, g, foot)

    monkeypatch.setattr(sl, "trace_feet", flipped)
    ts, Ws, _, _ = _run_landau(60, lomac=False)
    assert Ws[-1] > Ws[0]


def test_without_lomac_conservation_is_lost():
    """Without the correction mass/energy drift well above the Newton tolerance
    (Sec. 4.1 reports O(1e-4) for strong Landau)."""
    ts, Ws, tot0, tot1 = _run_landau(20, lomac=False)
    assert abs(tot1[0] - tot0[0]) / tot0[0] > 1e-10


@pytest.mark.parametrize("lomac", [True])
def test_2d2v_conservation_small(lomac):
    """2D-2V Landau on a 12^4 grid: DIRK3 start-up then BDF3; conservation at the Newton
    tolerance over four steps."""
    w = inputs.landau_2d2v(n=12, alpha=0.05, eps=1e-5, cap=12, dt=0.2)
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap, lomac=lomac)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)
    tot0 = stepper.totals(st, g)
    for _ in range(4):
        s = stepper.sl_step(st, w.dt, g, prm)
        assert s.converged
    tot1 = stepper.totals(st, g)
    assert abs(tot1[0] - tot0[0]) <= 1e-12 * tot0[0]
    assert abs(tot1[-1] - tot0[-1]) <= 1e-12 * tot0[-1]
    assert np.all(np.abs(tot1[1:3] - tot0[1:3]) <= 1e-12 * tot0[0])


@pytest.mark.slow
def test_bump_on_tail_2d2v_linear_damping():
    """2D-2V bump-on-tail data (Sec. 4.2 example; total density 1) at a small perturbation
    (alpha 0.01): the cos(k x1) cos(k x2) perturbation holds the wave vectors (k, +-k),
    |K| = 0.3 sqrt(2), along which the data reduce to a unit-temperature bulk of density
    17/20 and a beam of density 3/20, temperature 2.4 and drift 4.5 / sqrt(2).  That
    distribution has no unstable root at |K|; the electric energy follows its least-damped
    root, Im w = -0.1155 (Re w = 1.128): the rate fitted to the peaks of sqrt(W) on
    t in [2, 20] agrees within 2 %."""
    w = inputs.bump_on_tail_2d2v(N=(16, 16, 32, 32), alpha=0.01, eps=1e-6, cap=24, dt=0.2)
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)
    tot0 = stepper.totals(st, g)
    ts, Ws = [], []
    for _ in range(100):
        s = stepper.sl_step(st, w.dt, g, prm)
        assert s.converged
        ts.append(st.t)
        Ws.append(s.W)
    K = 0.3 * math.sqrt(2.0)
    root = dispersion.root(K, 1.1 - 0.1j, species=((17 / 20, 0.0, 1.0), (3 / 20, 4.5 / math.sqrt(2.0), 2.4)))
    assert abs(dispersion.dielectric(K, root, ((17 / 20, 0.0, 1.0), (3 / 20, 4.5 / math.sqrt(2.0), 2.4)))) < 1e-12
    rate, npk = _fit_rate(np.array(ts), np.array(Ws))
    assert npk >= 5
    assert abs(rate - root.imag) <= 0.02 * abs(root.imag), (rate, root)
    tot1 = stepper.totals(st, g)
    assert abs(tot1[0] - tot0[0]) <= 1e-12 * tot0[0]
    assert np.all(np.abs(tot1[1:3] - tot0[1:3]) <= 1e-12 * tot0[0])
    assert abs(tot1[3] - tot0[3]) <= 1e-12 * tot0[3]


def test_bump_on_tail_2d2v_mirror_symmetry():
    """The 2D-2V bump-on-tail data are even under (x2, v2) -> (-x2, -v2), which maps the
    cell-centred periodic grid onto itself (index j -> N - 1 - j), and the Vlasov-Poisson
    flow keeps that symmetry.  The cross approximation and the truncation of a SLAR call
    are not themselves mirror-symmetric and may each break it by about eps, so after one
    DIRK3 step (nine SLAR calls, ranks below the cap) f and its mirror image agree within
    9 eps; the v2 momentum stays zero."""
    w = inputs.bump_on_tail_2d2v(N=(8, 8, 16, 16), alpha=0.04, eps=1e-8, cap=32, dt=0.2)
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)
    s = stepper.sl_step(st, w.dt, g, prm)
    assert s.converged and max(s.aca_ranks) < w.rank_cap
    from oracle import ht as htmod
    f = htmod.densify(st.F)
    mirror = f[:, ::-1, :, ::-1]
    assert np.linalg.norm(f - mirror) <= 9 * w.eps * np.linalg.norm(f)
    assert abs(stepper.totals(st, g)[2]) <= 1e-12 * stepper.totals(st, g)[0]
    # not trivially symmetric in the other pair: the beam drifts along v1
    assert np.linalg.norm(f - f[:, :, ::-1, :]) > 1e-3 * np.linalg.norm(f)
