"""The C-ABI boundary beyond the hot-path parity: the moment selection mask, checkpoint and
bit-exact resume, and the error paths (SLAR_ENAN, SLAR_ENOCONV with the preconditioned and
learned solves falling back to plain JFNK, SLAR_EINVAL for replayed pivots outside the
matricisation, SLAR_ERANK when a rank cap binds with eps unmet).  Every failure is made on
the host (a NaN written into the conserved variables, a Newton cap of one iteration, bad
pivots, a tiny cap); nothing faults or hangs the GPU."""
import os

import numpy as np
import pytest
import torch

import convert
from oracle import field, sl
from oracle import ht as htmod
from paper_2606_29027_b300 import inputs, slar

pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _ctx(w, **kw):
    ctx = slar.Context(slar.make_config(w, **kw))
    ctx.init_ht(inputs.initial_factors(w))
    return ctx


# ---------------------------------------------------------------- moments mask

@pytest.mark.parametrize("w", [inputs.landau_1d1v(N=(32, 64), alpha=0.2),
                               inputs.landau_2d2v(n=16, alpha=0.2, eps=1e-6, cap=12)])
@pytest.mark.parametrize("mask", [slar.SLAR_MOM_M0, slar.SLAR_MOM_M1, slar.SLAR_MOM_M2, slar.SLAR_MOM_FLUX,
                                  slar.SLAR_MOM_M0 | slar.SLAR_MOM_M2, slar.SLAR_MOM_M1 | slar.SLAR_MOM_FLUX,
                                  slar.SLAR_MOM_ALL])
def test_moments_mask_selects_rows(w, mask):
    ctx = _ctx(w)
    ctx.step(w.dt)          # the state then carries a LoMaC correction
    full = torch.zeros((ctx.n_mom, ctx.NX), dtype=torch.float64, device="cuda")
    ctx.moments(full)
    dv = w.dv
    rows = []
    if mask & slar.SLAR_MOM_M0:
        rows += [0]
    if mask & slar.SLAR_MOM_M1:
        rows += list(range(1, 1 + dv))
    if mask & slar.SLAR_MOM_M2:
        rows += [1 + dv]
    if mask & slar.SLAR_MOM_FLUX:
        rows += list(range(dv + 2, ctx.n_mom))
    sel = torch.full((len(rows), ctx.NX), np.nan, dtype=torch.float64, device="cuda")
    ctx.moments(sel, mask)
    assert torch.equal(sel, full[rows])
    # and the full table is the oracle's
    h = convert.from_lib(ctx.export())
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    want = field.moments(h, g)
    assert np.linalg.norm(full.cpu().numpy() - want) <= 1e-12 * np.linalg.norm(want)


def test_moments_mask_rejects_unknown_bits():
    ctx = _ctx(inputs.landau_1d1v(N=(16, 32)))
    out = torch.zeros((5, ctx.NX), dtype=torch.float64, device="cuda")
    with pytest.raises(slar.SlarError) as e:
        ctx.moments(out, 16)
    assert e.value.status == slar.SLAR_EINVAL


# ---------------------------------------------------------------- checkpoint / restore

def _export_arrays(ctx):
    ex = ctx.export()
    arrs = list(ex["U"]) + [ex["Broot"]]
    for k in ("B12", "B34", "dC", "qv"):
        if ex.get(k) is not None:
            arrs.append(ex[k])
    U = torch.zeros((ctx.cfg.dv + 2, ctx.NX), dtype=torch.float64, device="cuda")
    ctx.get_conserved(U)
    return arrs + [U.cpu().numpy()]


@pytest.mark.parametrize("w,k_save", [(inputs.landau_1d1v(N=(32, 64), alpha=0.2, eps=1e-6, cap=16), 1),
                                      (inputs.landau_1d1v(N=(32, 64), alpha=0.2, eps=1e-6, cap=16), 3),
                                      (inputs.landau_2d2v(n=16, alpha=0.1, eps=1e-6, cap=12), 3)])
def test_resume_is_bit_exact(w, k_save, tmp_path):
    """FP64: run k_save steps, checkpoint, go on 3 steps; a fresh context restored from the
    checkpoint and stepped 3 times gives the same state bit for bit (k_save = 1 resumes in
    the middle of the DIRK3 start-up, 3 in BDF3 with its two-step history)."""
    path = str(tmp_path / "run.ckpt")
    a = _ctx(w, autotune=False)
    for _ in range(k_save):
        a.step(w.dt)
    a.checkpoint(path)
    Wa = [a.step(w.dt).field_energy for _ in range(3)]
    b = slar.Context(slar.make_config(w, autotune=False))
    b.restore(path)
    Wb = [b.step(w.dt).field_energy for _ in range(3)]
    assert Wa == Wb
    for x, y in zip(_export_arrays(a), _export_arrays(b)):
        assert x.shape == y.shape and np.array_equal(x, y)


def test_restore_rejects_other_grid_and_garbage(tmp_path):
    w = inputs.landau_1d1v(N=(32, 64), alpha=0.2)
    path = str(tmp_path / "a.ckpt")
    a = _ctx(w)
    a.checkpoint(path)
    other = slar.Context(slar.make_config(inputs.landau_1d1v(N=(32, 32), alpha=0.2)))
    with pytest.raises(slar.SlarError) as e:
        other.restore(path)
    assert e.value.status == slar.SLAR_EINVAL
    bad = str(tmp_path / "bad.ckpt")
    with open(bad, "wb") as f:
        f.write(b"not a checkpoint at all" * 10)
    with pytest.raises(slar.SlarError):
        a.restore(bad)
    with open(bad, "wb") as f:
        f.write(open(path, "rb").read()[:300])     # truncated
    with pytest.raises(slar.SlarError):
        slar.Context(slar.make_config(w)).restore(bad)
    with pytest.raises(slar.SlarError):
        a.restore(str(tmp_path / "missing.ckpt"))


def test_checkpoint_carries_network_parameters(tmp_path):
    w = inputs.landau_1d1v(N=(32, 64), alpha=0.2)
    m = w.dv + 2
    net_a = slar.Net(m, w.N[0], 1, hidden=8, max_batch=2)
    theta = np.random.default_rng(5).standard_normal(net_a.np).astype(np.float32) * 0.01
    net_a.set_params(theta)
    a = _ctx(w, solver="learned")
    a.attach_net(net_a)
    path = str(tmp_path / "net.ckpt")
    a.checkpoint(path)
    net_b = slar.Net(m, w.N[0], 1, hidden=8, max_batch=2)
    b = slar.Context(slar.make_config(w, solver="learned"))
    b.attach_net(net_b)
    b.restore(path)
    assert np.array_equal(net_b.get_params(), theta)


# ---------------------------------------------------------------- error paths

def test_nan_in_conserved_variables_gives_enan():
    w = inputs.landau_1d1v(N=(32, 64), alpha=0.2)
    ctx = _ctx(w)
    for _ in range(3):
        ctx.step(w.dt)
    U = torch.zeros((w.dv + 2, ctx.NX), dtype=torch.float64, device="cuda")
    n_i = ctx.get_conserved(U)
    Ubad = U.clone()
    Ubad[2, 5] = float("nan")
    ctx.set_conserved(Ubad, n_i)
    with pytest.raises(slar.SlarError) as e:
        ctx.step(w.dt)
    assert e.value.status == slar.SLAR_ENAN
    # the context stays usable: with finite data again the next step converges
    ctx.set_conserved(U, n_i)
    s = ctx.step(w.dt)
    assert s.converged


@pytest.mark.parametrize("solver", ["plain", "precond", "learned"])
def test_newton_cap_gives_enoconv_and_fallback(solver):
    """newton_max = 1 cannot reach the 1e-12 Newton tolerance: the step returns
    SLAR_ENOCONV; the preconditioned and learned solves report that they fell back to
    plain JFNK from U(F*) at the first BDF3 step, and the next BDF3 step is solved by plain
    JFNK alone (the preconditioned solve is switched off after a fallback)."""
    w = inputs.landau_1d1v(N=(32, 64), alpha=0.3)
    ctx = _ctx(w, solver=solver, newton_max=1)
    if solver == "learned":
        net = slar.Net(w.dv + 2, w.N[0], 1, hidden=8, max_batch=2)
        ctx.attach_net(net)
    statuses, fallbacks, built = [], [], []
    for _ in range(4):
        s = ctx.step(w.dt)
        statuses.append(s.status)
        fallbacks.append(s.fallback)
        built.append(s.pc_built)
    assert statuses[-1] == slar.SLAR_ENOCONV
    if solver != "plain":
        assert fallbacks[2] and built[2]   # first BDF3 step: preconditioned solve, then plain JFNK
        assert not fallbacks[3] and not built[3]   # next BDF3 step: plain JFNK only


def test_replayed_pivots_outside_the_matricisation_are_rejected():
    w = inputs.landau_1d1v(N=(32, 64), alpha=0.2)
    ctx = _ctx(w)
    E = torch.zeros((1, ctx.NX), dtype=torch.float64, device="cuda")
    ctx.set_pivot_replay([[(0, 3), (40, 5)]])      # row 40 >= M1 = 32
    with pytest.raises(slar.SlarError) as e:
        ctx.advect(0.1, E)
    assert e.value.status == slar.SLAR_EINVAL
    ctx.set_pivot_replay([[(0, 64)]])               # column 64 >= M2 = 64
    with pytest.raises(slar.SlarError) as e:
        ctx.advect(0.1, E)
    assert e.value.status == slar.SLAR_EINVAL


def test_rank_cap_with_eps_unmet_gives_erank():
    """A cap of 2 with eps 1e-12: the cross approximation stops at the cap with its stop test
    unmet -> SLAR_ERANK (a warning: the step completes and conserves)."""
    w = inputs.landau_1d1v(N=(32, 64), alpha=0.3, eps=1e-12, cap=2)
    ctx = _ctx(w)
    s = ctx.step(w.dt)
    assert s.status == slar.SLAR_ERANK and s.rank_capped > 0 and s.converged
    # truncation: a random rank-6 state truncated to cap 2 at eps 1e-12
    h = htmod.from_raw(inputs.random_ht((32, 64), (6, 6), 3))
    ctx.import_ht(**convert.to_lib(h))
    ctx.truncate(1e-12, 2)
    assert ctx.last_status == slar.SLAR_ERANK
    ctx.truncate(1e-1, 64)
    assert ctx.last_status == slar.SLAR_OK
