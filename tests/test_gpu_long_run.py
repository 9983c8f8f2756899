"""Long-horizon GPU parity on the 1D-1V weak Landau workload (x in [0, 4 pi), N_x = 64;
v in [-6, 6], N_v = 128; alpha 0.01, k 0.5; rank cap 16, eps 1e-6, dt 0.1, Newton
tolerance 1e-12; 200 steps = t = 20), Sec. 4.1 weak Landau damping example.

* With the oracle's pivots replayed (every one of the 612 SLAR calls: 2 DIRK3 start-up
  steps of 9 calls, then 198 BDF3 steps of 3), the FP64 GPU run reproduces the oracle's
  electric-energy history to 1e-8 relative and the final f and U to 1e-9.
* Free-running (the GPU picks its own pivots), the damping rate fitted to the peaks of
  sqrt(W) on t in [2, 20] is within 2 % of the linear root (-0.1533 at k = 0.5), and
  mass, momentum and energy of U stay at their initial values to 1e-12 relative
  (momentum relative to the mass, its initial value being zero).
"""
import numpy as np
import pytest
import torch

import convert
from oracle import dispersion, sl, stepper
from oracle import ht as htmod
from paper_2606_29027_b300 import inputs, slar

pytestmark = pytest.mark.gpu

STEPS = 200


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def fit_rate(ts, Ws, t0=2.0, t1=20.0):
    A = np.sqrt(np.asarray(Ws))
    ts = np.asarray(ts)
    pk = [i for i in range(1, len(A) - 1) if A[i] > A[i - 1] and A[i] >= A[i + 1] and t0 <= ts[i] <= t1]
    return np.polyfit(ts[pk], np.log(A[pk]), 1)[0], len(pk)


@pytest.fixture(scope="module")
def oracle_run():
    w = inputs.landau_1d1v()
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap, newton_tol=w.newton_tol)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)
    Ws, pivots = [], []
    for _ in range(STEPS):
        s = stepper.sl_step(st, w.dt, g, prm)
        assert s.converged
        Ws.append(s.W)
        pivots += s.pivots
    return w, g, st, np.array(Ws), pivots


def _gpu_run(w, pivots=None):
    ctx = slar.Context(slar.make_config(w))
    ctx.init_ht(inputs.initial_factors(w))
    if pivots is not None:
        ctx.set_pivot_replay(pivots)
    Ws, tots = [], []
    U = torch.zeros((w.dv + 2, ctx.NX), dtype=torch.float64, device="cuda")
    ctx.get_conserved(U)
    cell = (w.hi[0] - w.lo[0]) / w.N[0]
    tot0 = U.sum(dim=1).cpu().numpy() * cell
    for _ in range(STEPS):
        s = ctx.step(w.dt)
        assert s.converged and s.status in (slar.SLAR_OK, slar.SLAR_ERANK)
        Ws.append(s.field_energy)
        tots.append(np.array(s.totals[: w.dv + 2]))
    ctx.get_conserved(U)
    return ctx, np.array(Ws), tot0, np.array(tots), U.cpu().numpy()


def test_replayed_run_matches_oracle_history(oracle_run):
    w, g, st, Wo, pivots = oracle_run
    assert len(pivots) == 2 * 9 + (STEPS - 2) * 3
    ctx, Wg, _, _, U = _gpu_run(w, pivots)
    assert relerr(Wg, Wo) < 1e-8
    assert relerr(U, st.U) < 1e-9
    got = htmod.densify(convert.from_lib(ctx.export()))
    assert relerr(got, htmod.densify(st.F)) < 1e-9


def test_free_running_rate_and_conservation(oracle_run):
    w = oracle_run[0]
    ctx, Wg, tot0, tots, _ = _gpu_run(w)
    ts = w.dt * np.arange(1, STEPS + 1)
    rate, npk = fit_rate(ts, Wg)
    root = dispersion.landau_rate(0.5).imag
    assert npk >= 4
    assert abs(rate - root) <= 0.02 * abs(root), (rate, root)
    mass0, mom0, en0 = tot0[0], tot0[1], tot0[2]
    drift = np.abs(tots - tot0[None, :])
    assert drift[:, 0].max() <= 1e-12 * abs(mass0)
    assert drift[:, 1].max() <= 1e-12 * abs(mass0)
    assert drift[:, 2].max() <= 1e-12 * abs(en0)
    assert abs(mom0) < 1e-12 * abs(mass0)
