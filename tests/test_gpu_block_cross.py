"""GPU block cross approximation (slar_config.aca_block = b > 1; the rank-level parallel
HTACA of the scope's "next" rows) against the oracle's block cross approximation, free-running
(the GPU chooses its own pivots): the same rank, the same number of sampled entries, the
reconstructed f to the FP64 bar 1e-9; full steps with blocks against the oracle's steps with
blocks (W to 1e-8, U and f to 1e-9).

The cases keep the ranks below the cap (an approximation cut by the cap has not reached eps,
and two valid pivot sequences can then differ far beyond it) and use eps >= 1e-5, where an
eigen-solver of absolute accuracy (the oracle's) resolves the kept eigenvectors to
u / sqrt(eps^2 / (2d - 3)) <= 1e-10 of ||F||."""
import math

import numpy as np
import pytest
import torch

import convert
from oracle import cross, sl, stepper
from oracle import ht as htmod
from paper_2606_29027_b300 import inputs, slar

import test_gpu_parity as P

pytestmark = pytest.mark.gpu


def _rank_decision_conditioning(entry_fn, N, eps, cap, b):
    """Smallest relative eigenvalue gap at a rank cut and smallest relative distance of the
    discarded tail from the threshold, over the nodes of the oracle's truncation of its
    block cross approximation: a threshold that splits a near-degenerate pair (gap ~1e-2)
    leaves the kept eigenvector to u ||G|| / gap for any solver of absolute accuracy."""
    half = len(N) // 2
    M1, M2 = int(np.prod(N[:half])), int(np.prod(N[half:]))
    left = np.stack(np.unravel_index(np.arange(M1), N[:half]), axis=1)
    right = np.stack(np.unravel_index(np.arange(M2), N[half:]), axis=1)
    rf = lambda rows: np.stack([entry_fn(np.concatenate([np.repeat(left[i:i + 1], M2, 0), right], 1)) for i in rows])
    cf = lambda cols: np.stack([entry_fn(np.concatenate([left, np.repeat(right[j:j + 1], M1, 0)], 1))
                                for j in cols], axis=1)
    res = cross.aca_block(rf, cf, M1, M2, eps, cap, b)
    h = htmod.orthogonalize(cross.embed(res["U"], res["V"], N))
    G = htmod.node_gramians(h)
    thr = eps ** 2 * float(np.sum(h.Broot ** 2)) / (2 * len(N) - 3)
    gap, margin = 1.0, 1.0
    for t, Gt in G.items():
        lam = np.sort(np.linalg.eigvalsh(Gt))[::-1]
        tail = np.concatenate([np.cumsum(lam[::-1])[::-1], [0.0]])
        k = int(np.argmax(tail <= thr))
        if 0 < k < len(lam):
            gap = min(gap, (lam[k - 1] - lam[k]) / lam[k - 1])
            margin = min(margin, abs(tail[k] - thr) / thr)
    return gap, margin


@pytest.mark.parametrize("b", [2, 4, 8])
@pytest.mark.parametrize("N", [(32, 64), (16, 16, 16, 16), (128, 128, 8, 8)])
def test_block_slar_call_matches_oracle(N, b):
    """A well-conditioned SLAR call (checked: every rank cut of the oracle's truncation has
    a relative eigenvalue gap above 10 % and a discarded tail more than 2 % away from the
    threshold)."""
    eps, cap = 1e-5, 64
    F0, g = P._landau_state(N, eps=1e-12, cap=24)
    dx = len(N) // 2
    E = inputs.random_field(N[:dx], dx, 0.05, seed=15)
    tau = 0.2
    fn = lambda idx: sl.sl_eval(F0, E, tau, idx, g)
    gap, margin = _rank_decision_conditioning(fn, N, eps, cap, b)
    assert gap > 0.1 and margin > 0.02
    want, info = cross.htaca(fn, N, eps, cap, return_info=True, block=b)
    lo, hi = P.box(N)
    cfg = slar.make_config(dx=dx, dv=dx, N=N, lo=lo, hi=hi, eps=eps, rank_cap=cap, aca_block=b)
    ctx = slar.Context(cfg)
    P.load(ctx, F0)
    k, nent = ctx.advect(tau, P.dev(E))
    assert k == info["aca_rank"] < min(cap, int(np.prod(N[:dx])), int(np.prod(N[dx:])))
    assert nent == info["entries"]
    got = htmod.densify(convert.from_lib(ctx.export()))
    assert P.relerr(got, htmod.densify(want)) < 1e-9


@pytest.mark.parametrize("b", [4])
@pytest.mark.parametrize("w", [inputs.landau_1d1v(N=(32, 64), alpha=0.05, eps=1e-6, cap=16),
                               inputs.landau_2d2v(n=16, alpha=0.05, eps=1e-5, cap=32)])
def test_block_steps_match_oracle(w, b):
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap, newton_tol=w.newton_tol, block=b)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)
    ctx = slar.Context(slar.make_config(w, aca_block=b))
    ctx.init_ht(inputs.initial_factors(w))
    Wg, Wo = [], []
    for _ in range(4):
        s = ctx.step(w.dt)
        so = stepper.sl_step(st, w.dt, g, prm)
        assert s.converged and so.converged
        assert list(s.aca_rank[: s.n_slar]) == so.aca_ranks
        Wg.append(s.field_energy)
        Wo.append(so.W)
    assert P.relerr(np.array(Wg), np.array(Wo)) < 1e-8
    U = torch.zeros((w.dv + 2, ctx.NX), dtype=torch.float64, device="cuda")
    ctx.get_conserved(U)
    assert P.relerr(U.cpu().numpy(), st.U) < 1e-9
    assert P.relerr(htmod.densify(convert.from_lib(ctx.export())), htmod.densify(st.F)) < 1e-9


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16x6"])
def test_block_reduced_precision_close_to_fp64(prec):
    """Blocks with FP32, BF16x3 and BF16x6 entries (the tensor-core evaluator evaluates a block of
    fibres per launch): SLAR calls within the precision bars of the one-fibre path."""
    N = (16, 16, 16, 16)
    eps, cap = 1e-5, 64
    F0, g = P._landau_state(N, eps=1e-12, cap=24)
    E = inputs.random_field(N[:2], 2, 0.1, seed=13)
    want, info = cross.htaca(lambda idx: sl.sl_eval(F0, E, 0.3, idx, g), N, eps, cap, block=4, return_info=True)
    assert info["aca_rank"] < cap
    lo, hi = P.box(N)
    cfg = slar.make_config(dx=2, dv=2, N=N, lo=lo, hi=hi, eps=eps, rank_cap=cap, aca_block=4, precision=prec)
    ctx = slar.Context(cfg)
    P.load(ctx, F0)
    ctx.advect(0.3, P.dev(E))
    got = htmod.densify(convert.from_lib(ctx.export()))
    assert P.relerr(got, htmod.densify(want)) < 3 * eps
