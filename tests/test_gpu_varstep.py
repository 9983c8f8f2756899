"""Variable-step BDF3 and the adaptive step-size rule on the GPU against the oracle
(Sec. 3.2.3: variable-step BDF3 for adaptive time stepping, with a step-ratio condition).

* A run with uneven steps (ratios up to 1.25) and the oracle's pivots replayed matches the
  oracle step by step: W to 1e-8, U and f to 1e-9.
* slar_cfl_dt gives the oracle's step (cfl / max_i(a_i / Delta_i), capped) to 1e-13 at the
  initial state and to the state's parity (1e-9) along an adaptive run, and the adaptive run (each step's size from the
  rule) tracks the oracle's adaptive run and conserves mass, momentum and energy to 1e-12.
* A step longer than 1.4877 times the previous one is rejected after the start-up."""
import numpy as np
import pytest
import torch

import convert
from oracle import sl, stepper
from oracle import ht as htmod
from paper_2606_29027_b300 import inputs, slar

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _oracle(w):
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap, newton_tol=w.newton_tol)
    return g, prm, stepper.init_state(inputs.initial_factors(w), g, prm)


@pytest.mark.parametrize("w", [inputs.landau_1d1v(N=(32, 64), alpha=0.2, eps=1e-6, cap=16),
                               inputs.landau_2d2v(n=16, alpha=0.05, eps=1e-5, cap=12)])
def test_uneven_steps_match_oracle(w):
    dts = [0.1, 0.1, 0.12, 0.15, 0.1, 0.08, 0.1]
    g, prm, st = _oracle(w)
    Wo, piv = [], []
    for dt in dts:
        s = stepper.sl_step(st, dt, g, prm)
        assert s.converged
        Wo.append(s.W)
        piv += s.pivots
    ctx = slar.Context(slar.make_config(w))
    ctx.init_ht(inputs.initial_factors(w))
    ctx.set_pivot_replay(piv)
    Wg = []
    for dt in dts:
        s = ctx.step(dt)
        assert s.converged
        Wg.append(s.field_energy)
    assert relerr(Wg, Wo) < 1e-8
    U = torch.zeros((w.dv + 2, ctx.NX), dtype=torch.float64, device="cuda")
    ctx.get_conserved(U)
    assert relerr(U.cpu().numpy(), st.U) < 1e-9
    assert relerr(htmod.densify(convert.from_lib(ctx.export())), htmod.densify(st.F)) < 1e-9


def test_adaptive_run_tracks_oracle_and_conserves():
    """Coarse x, fine v and a strong field, so that the field term of the rule decides and
    the step varies over the run."""
    w = inputs.landau_1d1v(N=(16, 128), alpha=0.5, eps=1e-6, cap=16)
    cfl, dt_max, steps = 2.0, 0.5, 10
    g, prm, st = _oracle(w)
    dto, Wo, piv = [], [], []
    for _ in range(steps):
        dt = stepper.cfl_dt(st, g, cfl, dt_max)
        s = stepper.sl_step(st, dt, g, prm)
        assert s.converged
        dto.append(dt)
        Wo.append(s.W)
        piv += s.pivots
    assert max(dto) / min(dto) > 1.05          # the step does vary
    ctx = slar.Context(slar.make_config(w))
    ctx.init_ht(inputs.initial_factors(w))
    ctx.set_pivot_replay(piv)
    U = torch.zeros((w.dv + 2, ctx.NX), dtype=torch.float64, device="cuda")
    ctx.get_conserved(U)
    cell = (w.hi[0] - w.lo[0]) / w.N[0]
    tot0 = U.sum(dim=1).cpu().numpy() * cell
    dtg, Wg = [], []
    for _ in range(steps):
        dt = ctx.cfl_dt(cfl, dt_max)
        s = ctx.step(dt)
        assert s.converged
        dtg.append(dt)
        Wg.append(s.field_energy)
        tot = np.array(s.totals[:3])
        assert abs(tot[0] - tot0[0]) <= 1e-12 * abs(tot0[0])
        assert abs(tot[1] - tot0[1]) <= 1e-12 * abs(tot0[0])
        assert abs(tot[2] - tot0[2]) <= 1e-12 * abs(tot0[2])
    # the step follows max |E| of the state, which inherits the state's FP64 parity (1e-9)
    assert np.max(np.abs(np.array(dtg) - np.array(dto)) / np.array(dto)) < 1e-9
    assert dtg[0] == pytest.approx(dto[0], rel=1e-13)   # initial state: identical data
    assert relerr(Wg, Wo) < 1e-8


def test_step_ratio_above_bound_is_rejected():
    w = inputs.landau_1d1v(N=(32, 64), alpha=0.2)
    ctx = slar.Context(slar.make_config(w))
    ctx.init_ht(inputs.initial_factors(w))
    for _ in range(3):
        ctx.step(0.1)
    with pytest.raises(slar.SlarError) as e:
        ctx.step(0.16)
    assert e.value.status == slar.SLAR_EINVAL
    s = ctx.step(0.148)
    assert s.converged
    assert ctx.cfl_dt(100.0, 10.0) == pytest.approx(1.4877 * 0.148, rel=1e-14)
