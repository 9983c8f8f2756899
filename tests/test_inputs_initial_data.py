"""The workloads' separable initial data equal the closed forms they stand for, evaluated
directly at every cell centre (Sec. 4 examples; the 2D-2V two-stream data of the benchmark
configuration have the streams along v1 only)."""
import math

import numpy as np
import pytest

from paper_2606_29027_b300 import inputs


def _centres(w):
    return [w.lo[m] + (np.arange(w.N[m]) + 0.5) * (w.hi[m] - w.lo[m]) / w.N[m] for m in range(w.d)]


def _check(w, f0):
    c = np.meshgrid(*_centres(w), indexing="ij")
    want = f0(*c)
    got = inputs.initial_dense(w)
    assert np.abs(got - want).max() <= 1e-14 * np.abs(want).max()


def test_landau_1d1v():
    w = inputs.landau_1d1v(N=(16, 32), alpha=0.3)
    _check(w, lambda x, v: (1 + 0.3 * np.cos(0.5 * x)) * np.exp(-v * v / 2) / math.sqrt(2 * math.pi))


def test_two_stream_1d1v():
    w = inputs.two_stream_1d1v(N=(16, 32))
    _check(w, lambda x, v: (1 + 1e-3 * np.cos(0.2 * x)) / math.sqrt(2 * math.pi)
           * (np.exp(-(v - 2.4) ** 2 / 2) + np.exp(-(v + 2.4) ** 2 / 2)))


def test_bump_on_tail_1d1v():
    n_p = 9 / (10 * math.sqrt(2 * math.pi))
    n_b = 2 / (10 * math.sqrt(2 * math.pi))
    w = inputs.bump_on_tail_1d1v(N=(16, 64))
    assert w.hi[0] == pytest.approx(20 * math.pi / 3) and (w.lo[1], w.hi[1]) == (-13.0, 13.0)
    _check(w, lambda x, v: (1 + 0.04 * np.cos(0.3 * x))
           * (n_p * np.exp(-v * v / 2) + n_b * np.exp(-(v - 4.5) ** 2 / (2 * 0.5))))


def test_landau_2d2v():
    w = inputs.landau_2d2v(n=8, alpha=0.2)
    _check(w, lambda x1, x2, v1, v2: (1 + 0.2 * (np.cos(0.5 * x1) + np.cos(0.5 * x2)))
           * np.exp(-(v1 * v1 + v2 * v2) / 2) / (2 * math.pi))


def test_two_stream_2d2v():
    w = inputs.two_stream_2d2v(n=8)
    _check(w, lambda x1, x2, v1, v2: (1 + 0.005 * (np.cos(0.2 * x1) + np.cos(0.2 * x2))) / (4 * math.pi)
           * (np.exp(-(v1 - 2.4) ** 2 / 2) + np.exp(-(v1 + 2.4) ** 2 / 2)) * np.exp(-v2 * v2 / 2))


def test_bump_on_tail_2d2v():
    """Sec. 4.2 example with the densities normalised to total density 1 (n_p 2 pi +
    n_b 2 pi v_t = 1; the reading drops the printed overall factor)."""
    vt = 2.4
    n_p = 17 / (40 * math.pi)
    n_b = 3 / (40 * math.pi * vt)
    assert n_p * 2 * math.pi + n_b * 2 * math.pi * vt == pytest.approx(1.0, rel=1e-15)
    w = inputs.bump_on_tail_2d2v(N=(8, 8, 16, 16))
    assert w.hi[0] == pytest.approx(20 * math.pi / 3) and (w.lo[2], w.hi[2]) == (-13.0, 13.0)
    _check(w, lambda x1, x2, v1, v2: (1 + 0.04 * np.cos(0.3 * x1) * np.cos(0.3 * x2))
           * (n_p * np.exp(-(v1 * v1 + v2 * v2) / 2) + n_b * np.exp(-((v1 - 4.5) ** 2 + v2 * v2) / (2 * vt))))
