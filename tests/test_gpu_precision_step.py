"""One full BDF3 step in reduced precision against the FP64 step on the reconstructed f.
The GPU contexts start from the oracle's state after the two DIRK3 start-up steps (restored
from the library's checkpoint format) and replay the oracle's pivots of the step, so that
rounding alone separates the precisions: the cross approximations sample the same fibres in
every run, and the HSVD truncation and the LoMaC solve stay FP64.

Why one step, and ranks below the cap: each SLAR call truncates at eps, and a relative
perturbation u of its sampled entries moves the truncated tensor by a multiple of u that
depends on the conditioning of the pivots (measured with the oracle itself: 1e-7 noise on
the entries moves f by ~5e-7 per call on 2D-2V Landau 16^4 at eps 1e-6 with ranks below the
cap, ~2e-6 when the root rank sits at the cap); differences between precisions compound over
the calls of a run.

The step amplifies entry errors erratically: the oracle's own step, its entries perturbed by
absolute noise of one FP32 ulp (2^-23) of each call's largest entry, moves f by 2.3e-6 -
4.0e-6 (1D-1V Landau 32 x 64), 1.5e-5 - 9.3e-4 (2D-2V Landau 16^4) and 1.3e-5 - 1.2e-4
(two-stream 16^4) over three noise seeds; relative noise of 2^-22 moved the 1D-1V step by
1.5e-6 for one seed and by 8.4e-4 for another.  The FP32 entries themselves agree with the
FP64 ones to 0.9e-7 - 1.4e-7 (relative L2 over the grid).

Bars: FP64 GPU vs the oracle 1e-9 (relative L2 on f); FP32 entries vs the FP64 GPU step 3e-5
(measured 1.9e-5, 1D-1V); BF16x6 entries (six BF16 products, ~2^-24 relative per product,
but summed over K terms of mixed sign, and the root contraction on the tensor cores too:
their entry error against the oracle is up to 2.1x the FP32 evaluator's, 1.56e-6 against
7.35e-7 at rank 64) 3e-5 as well; BF16x3 entries (three BF16 products, ~2^-16 relative per
product) vs FP64 three times the oracle's own step response to 2^-16 relative noise on its
entries."""
import numpy as np
import pytest

import ckpt
import convert
from oracle import sl, stepper
from oracle import ht as htmod
from paper_2606_29027_b300 import inputs, slar

pytestmark = pytest.mark.gpu

BF16X3_NOISE = 2.0 ** -16


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


WORKLOADS = [inputs.landau_1d1v(N=(32, 64), alpha=0.2, eps=1e-6, cap=16),
             inputs.landau_2d2v(n=16, alpha=0.1, eps=1e-6, cap=32),
             inputs.two_stream_2d2v(n=16, eps=1e-6, cap=12)]


def _noisy_step(w, g, prm, st, pivots, noise, seed=11):
    """The oracle's step with every sampled entry multiplied by (1 + noise N(0, 1)): a
    perturbation planted in the oracle (on the CPU) to measure its sensitivity."""
    orig = sl.sl_eval
    rng = np.random.default_rng(seed)

    def noisy(*a, **k):
        v = orig(*a, **k)
        return v * (1.0 + noise * rng.standard_normal(np.shape(v)))

    sl.sl_eval = noisy
    try:
        s = stepper.sl_step(st, w.dt, g, prm, pivots=pivots)
    finally:
        sl.sl_eval = orig
    assert s.converged
    return htmod.densify(st.F)


@pytest.fixture(scope="module", params=range(len(WORKLOADS)), ids=[w.name for w in WORKLOADS])
def oracle_step(request, tmp_path_factory):
    import copy
    w = WORKLOADS[request.param]
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap, newton_tol=w.newton_tol)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)
    for _ in range(2):
        assert stepper.sl_step(st, w.dt, g, prm).converged
    path = str(tmp_path_factory.mktemp("ckpt") / f"{w.name}.ckpt")
    ckpt.write_checkpoint(path, w, st)
    st_noisy = copy.deepcopy(st)
    s = stepper.sl_step(st, w.dt, g, prm)
    assert s.converged
    f = htmod.densify(st.F)
    sens = relerr(_noisy_step(w, g, prm, st_noisy, s.pivots, BF16X3_NOISE), f)
    return w, path, s.pivots, f, sens


def _gpu_f(w, prec, path, pivots):
    ctx = slar.Context(slar.make_config(w, precision=prec))
    ctx.restore(path)
    ctx.set_pivot_replay(pivots)
    s = ctx.step(w.dt)
    assert s.converged
    f = htmod.densify(convert.from_lib(ctx.export()))
    ctx.close()
    return f


def test_fp64_step_matches_oracle(oracle_step):
    w, path, pivots, f_oracle, _ = oracle_step
    err = relerr(_gpu_f(w, "fp64", path, pivots), f_oracle)
    print(f"{w.name} fp64 vs oracle: {err:.2e}")
    assert err < 1e-9


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16x6"])
def test_reduced_precision_f_matches_fp64_step(oracle_step, prec):
    w, path, pivots, _, sens = oracle_step
    if prec.startswith("bf16") and w.dx == 1:
        pytest.skip("the tensor-core evaluator serves d = 4 trees (d = 2 uses the FP32 path)")
    f64 = _gpu_f(w, "fp64", path, pivots)
    fr = _gpu_f(w, prec, path, pivots)
    err = relerr(fr, f64)
    bar = {"fp32": 3e-5, "bf16x6": 3e-5, "bf16x3": 3.0 * sens}[prec]
    print(f"{w.name} {prec}: |f - f_fp64| / |f_fp64| = {err:.2e} (bar {bar:.2e}; oracle response to "
          f"2^-16 entry noise {sens:.2e})")
    assert err < bar
