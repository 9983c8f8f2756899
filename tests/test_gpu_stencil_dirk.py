"""GPU parity of the two higher-order options (the remark after Eq. tp_interp; Sec. 3.2.3's
DIRK coupling) against the FP64 oracle, through the C ABI.

* Quartic stencil (slar_config.interp_order = 4, FP64 entries): entries at the feet with
  and without the LoMaC correction (1e-12, as the quadratic evaluator), a SLAR call with the
  oracle's pivots (1e-9 on f) and full LoMaC steps (W 1e-8, U and f 1e-9).
* DIRK-only (SLAR_DIRK_ONLY): steps 3 and 4 (past the start-up, where BDF3 would take over)
  restored from the oracle's state and replaying its pivots, and a free run of four steps.
* Configurations the option excludes are rejected with SLAR_EINVAL.
"""
import numpy as np
import pytest
import torch

import ckpt
import convert
from oracle import cross, sl, stepper
from oracle import ht as htmod
from paper_2606_29027_b300 import inputs, slar

import test_gpu_parity as P

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _ctx(N, order=4, eps=1e-6, cap=16, **kw):
    lo, hi = P.box(N)
    d = len(N)
    cfg = slar.make_config(dx=d // 2, dv=d // 2, N=N, lo=lo, hi=hi, eps=eps, rank_cap=cap,
                           interp_order=order, **kw)
    return slar.Context(cfg), sl.PhaseGrid(d // 2, d // 2, N, lo, hi, order=order)


@pytest.mark.parametrize("N,ranks", P.CASES)
@pytest.mark.parametrize("with_corr", [False, True])
@pytest.mark.parametrize("foot", ["rk3", "euler"])
def test_quartic_entries_match_oracle(N, ranks, with_corr, foot):
    ctx, g = _ctx(N, foot=foot)
    h, dC, qv = P.rand_state(N, ranks, 3, with_corr)
    P.load(ctx, h, dC, qv)
    dx = len(N) // 2
    E = inputs.random_field(N[:dx], dx, 0.6, seed=4)
    idx = inputs.random_tuples(N, 3000 + 37, seed=5)
    out = torch.zeros(idx.shape[0], dtype=torch.float64, device="cuda")
    ctx.sl_eval(0.37, P.dev(E), P.dev(idx, torch.int32), out)
    want = sl.sl_eval(h, E, 0.37, idx, g, foot)
    assert relerr(out.cpu().numpy(), want) < 1e-12
    # the quadratic oracle is far from it: the order is in effect on the GPU
    g2 = sl.PhaseGrid(g.dx, g.dv, g.N, g.lo, g.hi)
    assert relerr(out.cpu().numpy(), sl.sl_eval(h, E, 0.37, idx, g2, foot)) > 1e-8
    ctx.close()


@pytest.mark.parametrize("N", [(32, 64), (16, 16, 16, 16)])
def test_quartic_slar_call_matches_oracle(N):
    eps, cap = 1e-7, 24
    F0, _ = P._landau_state(N, eps=1e-12, cap=cap)
    ctx, g = _ctx(N, eps=eps, cap=cap)
    dx = len(N) // 2
    E = inputs.random_field(N[:dx], dx, 0.3, seed=13)
    want, info = cross.htaca(lambda idx: sl.sl_eval(F0, E, 0.45, idx, g), N, eps, cap, return_info=True)
    P.load(ctx, F0)
    ctx.set_pivot_replay([info["pivots"]])
    k, _ = ctx.advect(0.45, P.dev(E))
    assert k == info["aca_rank"]
    assert relerr(htmod.densify(convert.from_lib(ctx.export())), htmod.densify(want)) < 1e-9
    ctx.close()


def _pair(w, steps, order=2, dirk_only=False, replay=True):
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi, order=order)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap, newton_tol=w.newton_tol, dirk_only=dirk_only)
    fac = inputs.initial_factors(w)
    st = stepper.init_state(fac, g, prm)
    ctx = slar.Context(slar.make_config(w, interp_order=order, dirk_only=dirk_only))
    ctx.init_ht(fac)
    Wo, piv = [], []
    for _ in range(steps):
        s = stepper.sl_step(st, w.dt, g, prm)
        assert s.converged
        Wo.append(s.W)
        piv += s.pivots
    if replay:
        ctx.set_pivot_replay(piv)
    Wg = []
    for _ in range(steps):
        s = ctx.step(w.dt)
        assert s.converged
        Wg.append(s.field_energy)
    U = torch.zeros((w.dv + 2, ctx.NX), dtype=torch.float64, device="cuda")
    ctx.get_conserved(U)
    f = htmod.densify(convert.from_lib(ctx.export()))
    ctx.close()
    return st, np.array(Wg), np.array(Wo), U.cpu().numpy(), f


@pytest.mark.parametrize("w", [inputs.landau_1d1v(N=(32, 64), alpha=0.05, eps=1e-6, cap=16),
                               inputs.landau_2d2v(n=16, alpha=0.05, eps=1e-5, cap=16)])
@pytest.mark.parametrize("replay", [True, False])
def test_quartic_steps_match_oracle(w, replay):
    """Four LoMaC steps (two DIRK3, two BDF3) with the quartic stencil."""
    st, Wg, Wo, U, f = _pair(w, 4, order=4, replay=replay)
    assert relerr(Wg, Wo) < 1e-8
    assert relerr(U, st.U) < 1e-9
    assert relerr(f, htmod.densify(st.F)) < 1e-9


@pytest.mark.parametrize("w", [inputs.landau_1d1v(N=(32, 64), alpha=0.2, eps=1e-6, cap=16),
                               inputs.landau_2d2v(n=16, alpha=0.05, eps=1e-5, cap=16)])
def test_dirk_only_steps_match_oracle(w, tmp_path):
    """Steps 3 and 4 in DIRK-only mode from the oracle's state after the start-up (restored
    from the checkpoint format), replaying the oracle's nine SLAR calls per step; then a
    free four-step run from the initial data."""
    import copy
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap, newton_tol=w.newton_tol, dirk_only=True)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)
    for _ in range(2):
        assert stepper.sl_step(st, w.dt, g, prm).converged
    path = str(tmp_path / "after_startup.ckpt")
    ckpt.write_checkpoint(path, w, st)
    Wo, piv = [], []
    for _ in range(2):
        s = stepper.sl_step(st, w.dt, g, prm)
        assert s.converged and len(s.pivots) == 9
        Wo.append(s.W)
        piv += s.pivots
    ctx = slar.Context(slar.make_config(w, dirk_only=True))
    ctx.restore(path)
    ctx.set_pivot_replay(piv)
    Wg = []
    for _ in range(2):
        s = ctx.step(w.dt)
        assert s.converged and s.n_slar == 9
        Wg.append(s.field_energy)
    assert relerr(Wg, Wo) < 1e-8
    U = torch.zeros((w.dv + 2, ctx.NX), dtype=torch.float64, device="cuda")
    ctx.get_conserved(U)
    assert relerr(U.cpu().numpy(), st.U) < 1e-9
    assert relerr(htmod.densify(convert.from_lib(ctx.export())), htmod.densify(st.F)) < 1e-9
    ctx.close()
    st2, Wg2, Wo2, U2, f2 = _pair(w, 4, dirk_only=True, replay=False)
    assert relerr(Wg2, Wo2) < 1e-8
    assert relerr(U2, st2.U) < 1e-9
    assert relerr(f2, htmod.densify(st2.F)) < 1e-9


def test_dirk_only_has_no_ratio_bound():
    w = inputs.landau_1d1v(N=(32, 64), alpha=0.1, eps=1e-6, cap=16)
    for dirk in (False, True):
        ctx = slar.Context(slar.make_config(w, dirk_only=dirk))
        ctx.init_ht(inputs.initial_factors(w))
        for _ in range(2):
            ctx.step(0.05)
        if dirk:
            assert ctx.step(0.2).converged          # ratio 4
            assert ctx.cfl_dt(50.0, 1.0) == 1.0      # no cap from the previous step
        else:
            with pytest.raises(RuntimeError):
                ctx.step(0.2)
        ctx.close()


@pytest.mark.parametrize("kw", [dict(precision="fp32"), dict(precision="bf16x3"), dict(order=3)])
def test_unsupported_orders_rejected(kw):
    N = (16, 16, 16, 16)
    lo, hi = P.box(N)
    order = kw.pop("order", 4)
    cfg = slar.make_config(dx=2, dv=2, N=N, lo=lo, hi=hi, interp_order=order, **kw)
    with pytest.raises(RuntimeError):
        slar.Context(cfg)
