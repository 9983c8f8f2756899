"""Learned JFNK warm start: a small periodic convolutional network on the spatial grid that
maps the macroscopic state of a step to an initial guess for the Newton solve and to a
per-point (dv+2) x (dv+2) block used inside the Krylov preconditioner.

Test infrastructure: part of the FP64 oracle, never called by the CUDA path.

This component is an addition to the paper's method (the paper solves the macroscopic
system of Sec. 3.2.3 by plain JFNK from U(F*)); the plain Newton iteration stays the judge
of the residual, so the network can only change how many iterations are needed.

Definitions (all arrays float64, channel-first, spatial grid n0 x n1, n1 = 1 in 1D):

* conv3x3: out[o, i, j] = b[o] + sum_c sum_{p,q in -1..1} W[o, c, p+1, q+1] x[c, i+p, j+q],
  indices periodic (a cross-correlation, as in most deep-learning libraries).
* network: h1 = tanh(conv(x)), h2 = tanh(conv(h1)), h3 = tanh(conv(h2)), y = conv(h3);
  channels 2m -> H -> H -> H -> m + m*m with m = dv + 2 and H hidden channels.
* features of a step (Sec. 3.2.3 quantities): the first m channels are the fluctuations of
  U^n about their spatial means (for Vlasov-Poisson electrons these are -rho, -J and the
  energy density e), each divided by its RMS over the grid; the last m channels are the
  kinetic increment U* - U^n (U* = moments of the SLAR state F*), each divided by its RMS.
* outputs: y[:m] is the scaled guess correction d, with U_guess = U* + s_D d (s_D the RMS
  scales of U* - U^n); y[m:] read row-major as b(x), the block is B(x) = I + b(x).
* losses, averaged over samples and points:
    L_guess = mean ||d - (U^{n+1} - U*) / s_D||^2,
    L_block = mean_s ||B(x) w_s(x) - v_s(x)||^2   (w_s = J P v_s, probe pairs),
  total L = L_guess + L_block.
* Adam (Kingma and Ba 2015, Algorithm 1) with bias-corrected moments.

Flat parameter layout (shared with the CUDA library's C interface): for layer l = 0..3,
W_l (Cout, Cin, 3, 3) row-major followed by b_l (Cout).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np

HIDDEN = 32
N_LAYERS = 4


def layer_shapes(m: int, hidden: int = HIDDEN) -> List[Tuple[int, int]]:
    """(Cout, Cin) of the four convolutions."""
    return [(hidden, 2 * m), (hidden, hidden), (hidden, hidden), (m + m * m, hidden)]


def n_params(m: int, hidden: int = HIDDEN) -> int:
    return sum(co * ci * 9 + co for co, ci in layer_shapes(m, hidden))


def unflatten(theta: np.ndarray, m: int, hidden: int = HIDDEN):
    """Split the flat parameter vector into [(W, b)] per layer."""
    out, off = [], 0
    for co, ci in layer_shapes(m, hidden):
        W = theta[off: off + co * ci * 9].reshape(co, ci, 3, 3)
        off += co * ci * 9
        b = theta[off: off + co]
        off += co
        out.append((W, b))
    assert off == theta.size
    return out


def flatten(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in layers])


def init_params(m: int, seed: int, hidden: int = HIDDEN) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases; the last layer is
    scaled by 0.1 so that the initial guess stays near U* and the block near I."""
    rng = np.random.default_rng(seed)
    layers = []
    shapes = layer_shapes(m, hidden)
    for l, (co, ci) in enumerate(shapes):
        a = 1.0 / np.sqrt(ci * 9)
        if l == len(shapes) - 1:
            a *= 0.1
        layers.append((rng.uniform(-a, a, size=(co, ci, 3, 3)), np.zeros(co)))
    return flatten(layers)


def conv3x3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Periodic 3x3 cross-correlation, x (Cin, n0, n1) -> (Cout, n0, n1)."""
    co = W.shape[0]
    out = np.empty((co,) + x.shape[1:])
    out[:] = b[:, None, None]
    for p in (-1, 0, 1):
        for q in (-1, 0, 1):
            # xs[c, i, j] = x[c, i + p, j + q]
            xs = np.roll(np.roll(x, -p, axis=1), -q, axis=2)
            out += np.einsum("oc,cij->oij", W[:, :, p + 1, q + 1], xs)
    return out


def conv3x3_grad_input(dy: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Adjoint of conv3x3 in its input: dx[c, i, j] = sum_o sum_pq W[o,c,p,q] dy[o, i-p, j-q]."""
    ci = W.shape[1]
    dx = np.zeros((ci,) + dy.shape[1:])
    for p in (-1, 0, 1):
        for q in (-1, 0, 1):
            t = np.einsum("oc,oij->cij", W[:, :, p + 1, q + 1], dy)
            dx += np.roll(np.roll(t, p, axis=1), q, axis=2)
    return dx


def conv3x3_grad_params(x: np.ndarray, dy: np.ndarray):
    """dW[o, c, p, q] = sum_ij dy[o, i, j] x[c, i+p, j+q]; db[o] = sum_ij dy[o, i, j]."""
    co, ci = dy.shape[0], x.shape[0]
    dW = np.zeros((co, ci, 3, 3))
    for p in (-1, 0, 1):
        for q in (-1, 0, 1):
            xs = np.roll(np.roll(x, -p, axis=1), -q, axis=2)
            dW[:, :, p + 1, q + 1] = np.einsum("oij,cij->oc", dy, xs)
    return dW, dy.sum(axis=(1, 2))


def forward(theta: np.ndarray, x: np.ndarray, m: int, hidden: int = HIDDEN):
    """Network output y (m + m^2, n0, n1) and the activations needed by backward."""
    layers = unflatten(theta, m, hidden)
    acts = [x]
    h = x
    for l, (W, b) in enumerate(layers):
        z = conv3x3(h, W, b)
        h = np.tanh(z) if l < len(layers) - 1 else z
        acts.append(h)
    return h, acts


def backward(theta: np.ndarray, acts, dy: np.ndarray, m: int, hidden: int = HIDDEN):
    """Gradient of a scalar loss with respect to the flat parameters, given dL/dy."""
    layers = unflatten(theta, m, hidden)
    grads = [None] * len(layers)
    g = dy
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        x_in = acts[l]
        dW, db = conv3x3_grad_params(x_in, g)
        grads[l] = (dW, db)
        if l > 0:
            g = conv3x3_grad_input(g, W) * (1.0 - acts[l] ** 2)   # tanh' = 1 - tanh^2
    return flatten(grads)


@dataclass
class Sample:
    """One training sample of a Newton solve: features x (2m, n0, n1), guess target
    t (m, n0, n1) and S probe pairs v, w (S, m, n0, n1)."""
    x: np.ndarray
    t: np.ndarray
    v: np.ndarray
    w: np.ndarray


def rms_scales(a: np.ndarray, floor: float) -> np.ndarray:
    """Per-channel RMS over the grid, floored (a: (m, NX))."""
    return np.maximum(np.sqrt(np.mean(a * a, axis=1)), floor)


SCALE_FLOOR = 1e-30


def features(Un: np.ndarray, Ustar: np.ndarray, shape2d: Tuple[int, int]):
    """Network input (2m, n0, n1) and the guess scales s_D (m,) from U^n and U* (m, NX)."""
    m = Un.shape[0]
    fl = Un - Un.mean(axis=1, keepdims=True)
    sU = rms_scales(fl, SCALE_FLOOR)
    dU = Ustar - Un
    sD = rms_scales(dU, SCALE_FLOOR)
    x = np.concatenate([fl / sU[:, None], dU / sD[:, None]]).reshape((2 * m,) + shape2d)
    return x, sD


def guess_from_output(y: np.ndarray, Ustar: np.ndarray, sD: np.ndarray) -> np.ndarray:
    m = Ustar.shape[0]
    return Ustar + sD[:, None] * y[:m].reshape(m, -1)


def apply_block(y: np.ndarray, v: np.ndarray) -> np.ndarray:
    """B(x) v(x) with B = I + b, b = y[m:] row-major (m, m) per point; v (m, NX)."""
    m = v.shape[0]
    b = y[m:].reshape(m, m, -1)
    return v + np.einsum("ijx,jx->ix", b, v)


def loss_and_grad_output(y: np.ndarray, smp: Sample):
    """Total loss of one sample and dL/dy."""
    m = smp.t.shape[0]
    npts = int(np.prod(smp.t.shape[1:]))
    dy = np.zeros_like(y)
    r = y[:m] - smp.t
    L_guess = float(np.sum(r * r)) / (m * npts)
    dy[:m] = 2.0 * r / (m * npts)
    S = smp.v.shape[0]
    b = y[m:].reshape(m, m, -1)
    L_block = 0.0
    db = np.zeros_like(b)
    for s in range(S):
        w = smp.w[s].reshape(m, -1)
        v = smp.v[s].reshape(m, -1)
        e = w + np.einsum("ijx,jx->ix", b, w) - v
        L_block += float(np.sum(e * e)) / (S * m * npts)
        db += 2.0 * np.einsum("ix,jx->ijx", e, w) / (S * m * npts)
    dy[m:] = db.reshape((m * m,) + y.shape[1:])
    return L_guess + L_block, dy


def loss(theta: np.ndarray, batch: List[Sample], m: int, hidden: int = HIDDEN) -> float:
    return float(np.mean([loss_and_grad_output(forward(theta, s.x, m, hidden)[0], s)[0]
                          for s in batch]))


def loss_grad(theta: np.ndarray, batch: List[Sample], m: int, hidden: int = HIDDEN):
    """Mean loss over the batch and its gradient."""
    L = 0.0
    g = np.zeros_like(theta)
    for s in batch:
        y, acts = forward(theta, s.x, m, hidden)
        Ls, dy = loss_and_grad_output(y, s)
        L += Ls
        g += backward(theta, acts, dy, m, hidden)
    return L / len(batch), g / len(batch)


@dataclass
class Adam:
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8


def adam_step(theta, grad, mom1, mom2, t: int, opt: Adam):
    """One Adam update (t counts from 1); returns new (theta, mom1, mom2)."""
    mom1 = opt.beta1 * mom1 + (1.0 - opt.beta1) * grad
    mom2 = opt.beta2 * mom2 + (1.0 - opt.beta2) * grad * grad
    mhat = mom1 / (1.0 - opt.beta1 ** t)
    vhat = mom2 / (1.0 - opt.beta2 ** t)
    return theta - opt.lr * mhat / (np.sqrt(vhat) + opt.eps), mom1, mom2
