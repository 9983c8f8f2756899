"""Pins of the oracle's warm-start network and block-circulant preconditioner against
facts outside themselves: the convolution theorem, adjoint identities, central
differences, Adam's closed-form first step, exact inversion of circulant operators and
agreement of the preconditioned Newton solve with the plain one."""
import math

import numpy as np
import pytest

from oracle import macro, net, precond, stepper, sl
from paper_2606_29027_b300 import inputs


def _conv_fft(x, W, b):
    """Periodic cross-correlation through the convolution theorem."""
    co, ci = W.shape[:2]
    n0, n1 = x.shape[1:]
    out = np.zeros((co, n0, n1))
    X = np.fft.fft2(x)
    for o in range(co):
        acc = np.zeros((n0, n1), complex)
        for c in range(ci):
            K = np.zeros((n0, n1))
            for p in (-1, 0, 1):
                for q in (-1, 0, 1):
                    K[p % n0, q % n1] += W[o, c, p + 1, q + 1]
            acc += X[c] * np.conj(np.fft.fft2(K))
        out[o] = np.real(np.fft.ifft2(acc)) + b[o]
    return out


@pytest.mark.parametrize("shape", [(7, 5), (8, 8), (6, 1), (3, 4)])
def test_conv_matches_convolution_theorem(shape):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3,) + shape)
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    np.testing.assert_allclose(net.conv3x3(x, W, b), _conv_fft(x, W, b), atol=1e-12)


def test_conv_adjoint_identities():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 6, 5))
    y = rng.standard_normal((4, 6, 5))
    W = rng.standard_normal((4, 3, 3, 3))
    Ax = net.conv3x3(x, W, np.zeros(4))
    # <A x, y> = <x, A^T y>
    assert np.vdot(Ax, y) == pytest.approx(np.vdot(x, net.conv3x3_grad_input(y, W)), rel=1e-12)
    # <A x, y> is linear in W: = <W, dW(x, y)>
    dW, db = net.conv3x3_grad_params(x, y)
    assert np.vdot(Ax, y) == pytest.approx(np.vdot(W, dW), rel=1e-12)
    np.testing.assert_allclose(db, y.sum(axis=(1, 2)), rtol=1e-13)


def _tiny_problem(m=3, hidden=4, shape=(5, 4), S=2, seed=3):
    rng = np.random.default_rng(seed)
    theta = net.init_params(m, seed, hidden)
    theta += 0.3 * rng.standard_normal(theta.size)       # leave the small-init regime
    smp = net.Sample(x=rng.standard_normal((2 * m,) + shape),
                     t=rng.standard_normal((m,) + shape),
                     v=rng.standard_normal((S, m) + shape),
                     w=rng.standard_normal((S, m) + shape))
    return theta, smp


def test_network_gradient_central_differences():
    m, hidden = 3, 4
    theta, smp = _tiny_problem(m, hidden)
    L, g = net.loss_grad(theta, [smp], m, hidden)
    rng = np.random.default_rng(4)
    idx = rng.choice(theta.size, size=40, replace=False)
    h = 1e-6
    for i in idx:
        tp = theta.copy()
        tp[i] += h
        tm = theta.copy()
        tm[i] -= h
        fd = (net.loss(tp, [smp], m, hidden) - net.loss(tm, [smp], m, hidden)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3 * np.max(np.abs(g))), (i, fd, g[i])


def test_output_loss_gradient_central_differences():
    m = 3
    theta, smp = _tiny_problem(m)
    rng = np.random.default_rng(5)
    y = rng.standard_normal((m + m * m,) + smp.t.shape[1:])
    L, dy = net.loss_and_grad_output(y, smp)
    h = 1e-6
    for flat in rng.choice(y.size, size=30, replace=False):
        e = np.zeros(y.size)
        e[flat] = h
        e = e.reshape(y.shape)
        fd = (net.loss_and_grad_output(y + e, smp)[0] - net.loss_and_grad_output(y - e, smp)[0]) / (2 * h)
        assert fd == pytest.approx(dy.reshape(-1)[flat], rel=1e-6, abs=1e-10)


def test_block_is_identity_plus_output():
    m = 4
    rng = np.random.default_rng(6)
    y = rng.standard_normal((m + m * m, 3, 2))
    v = rng.standard_normal((m, 6))
    Bv = net.apply_block(y, v)
    for px in range(6):
        B = np.eye(m) + y[m:].reshape(m * m, 6)[:, px].reshape(m, m)
        np.testing.assert_allclose(Bv[:, px], B @ v[:, px], rtol=1e-13)


def test_adam_first_step_and_constant_gradient():
    opt = net.Adam(lr=0.01)
    theta = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -3.0, 1e-3])
    th, m1, m2 = net.adam_step(theta, g, np.zeros(3), np.zeros(3), 1, opt)
    # bias correction makes the first step lr * g / (|g| + eps)
    np.testing.assert_allclose(th, theta - opt.lr * g / (np.abs(g) + opt.eps), rtol=1e-14)
    for t in range(2, 6):
        prev = th
        th, m1, m2 = net.adam_step(th, g, m1, m2, t, opt)
        np.testing.assert_allclose(prev - th, opt.lr * g / (np.abs(g) + opt.eps), rtol=1e-12)


def test_features_are_normalised():
    rng = np.random.default_rng(7)
    Un = 1.0 + 0.01 * rng.standard_normal((4, 64))
    Us = Un + 1e-4 * rng.standard_normal((4, 64))
    x, sD = net.features(Un, Us, (8, 8))
    xf = x.reshape(8, -1)
    np.testing.assert_allclose(np.sqrt(np.mean(xf ** 2, axis=1)), 1.0, rtol=1e-13)
    np.testing.assert_allclose(xf[:4].mean(axis=1), 0.0, atol=1e-13)
    np.testing.assert_allclose(net.guess_from_output(np.concatenate([xf[4:], np.zeros((16, 64))]), Us, sD),
                               Us + (Us - Un), rtol=1e-13)


def test_gauss_jordan_inverse():
    rng = np.random.default_rng(8)
    for m in (1, 3, 4):
        A = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
        np.testing.assert_allclose(precond.gauss_jordan_inverse(A), np.linalg.inv(A), rtol=1e-10, atol=1e-12)
    np.testing.assert_array_equal(precond.gauss_jordan_inverse(np.zeros((3, 3))), np.eye(3))


def _circulant_G(shape2d, rng):
    """A spatially invariant linear operator U -> U + c D_x (A U) + s M U with spectral
    derivative D_x along axis 0 and constant matrices A, M."""
    m = 3
    A = rng.standard_normal((m, m))
    M = rng.standard_normal((m, m))
    n0, n1 = shape2d
    k = np.fft.fftfreq(n0, d=1.0 / n0)

    def deriv(f):
        F = np.fft.fft(f.reshape(shape2d), axis=0)
        return np.real(np.fft.ifft(1j * k[:, None] * F, axis=0)).reshape(-1)

    def G(U):
        AU = A @ U
        return U + 0.3 * np.stack([deriv(AU[c]) for c in range(m)]) + 0.1 * (M @ U)

    return G, m


def test_circulant_preconditioner_inverts_invariant_operator():
    rng = np.random.default_rng(9)
    shape2d = (8, 4)
    G, m = _circulant_G(shape2d, rng)
    U = rng.standard_normal((m, 32))
    G0 = G(U)
    P = precond.circulant_blocks(G, U, G0, shape2d)
    v = rng.standard_normal((m, 32))
    # P J v = v up to the finite-difference error of the probes
    np.testing.assert_allclose(precond.apply_circulant(P, G(v) - G(np.zeros_like(v))), v, atol=1e-6)


def test_right_preconditioned_jfnk_linear_one_step():
    rng = np.random.default_rng(10)
    shape2d = (8, 4)
    Gl, m = _circulant_G(shape2d, rng)
    b = rng.standard_normal((m, 32))
    G = lambda U: Gl(U) - b
    U0 = np.zeros((m, 32))
    P = precond.circulant_blocks(G, U0, G(U0), shape2d)
    U, st = precond.jfnk_right(G, U0, 1e-6, 1e-4, lambda y: precond.apply_circulant(P, y))
    assert st.converged and st.krylov <= 2
    U2, st2 = precond.jfnk_right(G, U0, 1e-6, 1e-4, None)
    U3, st3 = macro.jfnk(G, U0, 1e-6, 1e-4)
    np.testing.assert_allclose(U2, U3, rtol=0, atol=1e-14)
    assert st2.krylov == st3.krylov and st2.krylov > st.krylov
    np.testing.assert_allclose(U, U3, atol=1e-6)


@pytest.mark.parametrize("mode", ["circulant", "learned"])
def test_preconditioned_step_matches_plain(mode):
    """The preconditioner and the network change the iteration, not the solution: the
    BDF3 steps agree with the plain JFNK to the Newton tolerance."""
    w = inputs.landau_1d1v(N=(16, 32), alpha=0.3)
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    theta = net.init_params(3, seed=11)
    res = {}
    for md in ("none", mode):
        prm = stepper.Params(eps=w.eps, cap=w.rank_cap, precond=md, net_theta=theta)
        st = stepper.init_state(inputs.initial_factors(w), g, prm)
        its = []
        for _ in range(5):
            s = stepper.sl_step(st, w.dt, g, prm)
            assert s.converged
            its.append(s.krylov)
        res[md] = (st.U.copy(), its)
    scale = np.max(np.abs(res["none"][0]))
    np.testing.assert_allclose(res[mode][0], res["none"][0], atol=1e-10 * scale)
    assert sum(res[mode][1][2:]) < sum(res["none"][1][2:])


def test_training_sample_shapes_and_probe_pairs():
    w = inputs.landau_1d1v(N=(16, 32), alpha=0.3)
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)
    rec = []
    rng = np.random.default_rng(12)
    for s in range(3):
        stepper.sl_step(st, w.dt, g, prm, record=rec if s == 2 else None,
                        probes=rng.choice([-1.0, 1.0], size=(2, 3, 16)))
    assert len(rec) == 1
    smp = rec[0]
    assert smp.x.shape == (6, 16, 1) and smp.t.shape == (3, 16, 1)
    assert smp.v.shape == smp.w.shape == (3, 3, 16, 1)
    # w = J P v with P the circulant inverse: for this nearly invariant operator w ~ v
    rel = np.linalg.norm(smp.w - smp.v) / np.linalg.norm(smp.v)
    assert rel < 0.5
