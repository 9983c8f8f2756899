"""GPU tests of the ensemble step (uneven runs advanced concurrently on their own streams)
and of the entry-evaluator autotuner, through the C ABI."""
import numpy as np
import pytest

from paper_2606_29027_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_29027_b300 import slar  # noqa: E402


def _contexts(ws, autotune=False, solver="precond"):
    ctxs = []
    for w in ws:
        c = slar.Context(slar.make_config(w, precision="fp32", solver=solver, autotune=autotune,
                                          own_stream=True))
        c.init_ht(inputs.initial_factors(w))
        ctxs.append(c)
    torch.cuda.synchronize()
    return ctxs


def _state(c, w):
    U = torch.zeros((w.dv + 2, c.NX), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(c.stream):
        c.get_conserved(U)
    torch.cuda.synchronize()
    return U.cpu().numpy()


def test_ensemble_step_equals_sequential_steps():
    ws = inputs.ensemble(n_runs=8, seed=3, sizes=(8, 16), cap_range=(4, 12))
    A = _contexts(ws)
    B = _contexts(ws)
    steps = 4
    sa = [slar.ensemble_step(A, [w.dt for w in ws], threads=4) for _ in range(steps)]
    sb = [[c.step(w.dt) for c, w in zip(B, ws)] for _ in range(steps)]
    for i, w in enumerate(ws):
        np.testing.assert_array_equal(_state(A[i], w), _state(B[i], w))
        for s in range(steps):
            assert sa[s][i].field_energy == sb[s][i].field_energy
            assert sa[s][i].converged
    for c in A + B:
        c.close()


def test_ensemble_rejects_shared_stream():
    ws = inputs.ensemble(n_runs=2, seed=4, sizes=(8,), cap_range=(4, 6))
    st = torch.cuda.Stream()
    ctxs = [slar.Context(slar.make_config(w), stream=st) for w in ws]
    for c, w in zip(ctxs, ws):
        c.init_ht(inputs.initial_factors(w))
    with pytest.raises(slar.SlarError):
        slar.ensemble_step(ctxs, [0.1, 0.1])
    for c in ctxs:
        c.close()


def test_autotuned_tile_agrees_with_fixed_tile():
    w = inputs.landau_2d2v(n=16, alpha=0.3, cap=12)
    res = {}
    for tune in (False, True):
        c = slar.Context(slar.make_config(w, precision="fp64", autotune=tune))
        c.init_ht(inputs.initial_factors(w))
        st = [c.step(w.dt) for _ in range(4)]
        res[tune] = (_state(c, w), [s.field_energy for s in st], [s.eval_tile for s in st])
        c.close()
    assert all(t == 32 for t in res[False][2])
    assert all(t in (16, 32, 64) for t in res[True][2])
    U0, U1 = res[False][0], res[True][0]
    # the tile changes the summation order of the root contraction only; cross pivots are
    # chosen with a relative tie band, so the two runs follow the same path and differ by
    # rounding amplified over the steps (the FP64 parity bar, 1e-9)
    assert np.max(np.abs(U0 - U1)) <= 1e-9 * np.max(np.abs(U0))
    np.testing.assert_allclose(res[True][1], res[False][1], rtol=1e-8)
