"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the benchmark.

This module only *describes* workloads and draws random numbers.  It holds none of
the SLAR method's arithmetic (no stencils, no feet, no contractions, no moments):
it samples analytic initial data at the cell centres of the phase-space grid and
produces seeded random hierarchical-Tucker factors, index tuples and field arrays.

Workloads follow the paper's test problems (Sec. 4): Landau damping
(Example 4.1, 1D-1V; its 2D-2V analogue), and the two-stream instability
(Example 4.2 in 1D-1V, Example 4.4 in 2D-2V).  All data are synthetic and
analytic; no dataset is involved.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict
from typing import List, Optional, Sequence

import numpy as np


@dataclass
class Workload:
    """A Vlasov-Poisson run: grid, tree, tolerances and separable initial data.

    ``terms`` lists separable terms of f0: f0 = sum_t prod_mu terms[t][mu](coord_mu),
    each factor given as (kind, params) and sampled at the cell centres by
    :func:`initial_factors`.  Dimension order is (x1..x_dx, v1..v_dv).
    """
    name: str
    dx: int
    dv: int
    N: tuple
    lo: tuple
    hi: tuple
    eps: float
    rank_cap: int
    dt: float
    steps: int
    terms: list
    newton_tol: float = 1e-12
    krylov_tol: float = 1e-4
    lomac: bool = True
    alpha: float = 0.0
    k: float = 0.0

    @property
    def d(self) -> int:
        return self.dx + self.dv

    def to_dict(self):
        out = asdict(self)
        return out


def _cell_centres(lo: float, hi: float, n: int) -> np.ndarray:
    # Sampling points of the initial data: the centres of n uniform cells on [lo, hi).
    h = (hi - lo) / n
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * h


def _factor(kind: str, params: dict, x: np.ndarray) -> np.ndarray:
    if kind == "const":
        return np.full_like(x, params["c"])
    if kind == "cos":          # c * cos(k x)
        return params.get("c", 1.0) * np.cos(params["k"] * x)
    if kind == "maxwell":      # exp(-(x-u)^2 / (2 T)) / sqrt(2 pi T) * c
        u = params.get("u", 0.0)
        T = params.get("T", 1.0)
        c = params.get("c", 1.0)
        return c * np.exp(-((x - u) ** 2) / (2.0 * T)) / math.sqrt(2.0 * math.pi * T)
    if kind == "two_stream":   # c * (exp(-(x-u)^2/2) + exp(-(x+u)^2/2))
        u = params["u"]
        c = params.get("c", 1.0)
        return c * (np.exp(-((x - u) ** 2) / 2.0) + np.exp(-((x + u) ** 2) / 2.0))
    raise ValueError(f"unknown factor kind {kind!r}")


def initial_factors(w: Workload) -> List[List[np.ndarray]]:
    """Sample every separable factor of f0 at the cell centres: [term][mu] -> float64[N_mu]."""
    grids = [_cell_centres(w.lo[m], w.hi[m], w.N[m]) for m in range(w.d)]
    out = []
    for term in w.terms:
        out.append([_factor(kind, params, grids[m]) for m, (kind, params) in enumerate(term)])
    return out


def initial_dense(w: Workload) -> np.ndarray:
    """Dense f0 on the full grid (only for tiny grids)."""
    fac = initial_factors(w)
    F = None
    for term in fac:
        t = term[0]
        for f in term[1:]:
            t = np.multiply.outer(t, f)
        F = t if F is None else F + t
    return F


# --------------------------------------------------------------------------------------
# The five workloads of the benchmark family (1D-1V / 2D-2V Landau and two-stream).
# --------------------------------------------------------------------------------------

def landau_1d1v(N=(64, 128), alpha=0.01, k=0.5, vmax=6.0, eps=1e-6, cap=16, dt=0.1,
                steps=200) -> Workload:
    L = 2.0 * math.pi / k
    terms = [[("const", {"c": 1.0}), ("maxwell", {})],
             [("cos", {"k": k, "c": alpha}), ("maxwell", {})]]
    return Workload(name=f"landau_1d1v_{N[0]}x{N[1]}", dx=1, dv=1, N=tuple(N),
                    lo=(0.0, -vmax), hi=(L, vmax), eps=eps, rank_cap=cap, dt=dt,
                    steps=steps, terms=terms, alpha=alpha, k=k)


def bump_on_tail_1d1v(N=(64, 128), alpha=0.04, k=0.3, u=4.5, vt=0.5, vmax=13.0, eps=1e-5, cap=16,
                      dt=0.1, steps=200) -> Workload:
    # f0 = (1 + alpha cos kx)(n_p exp(-v^2/2) + n_b exp(-(v-u)^2/(2 vt))),
    # n_p = 9/(10 sqrt(2 pi)), n_b = 2/(10 sqrt(2 pi)); the bulk and the beam are separate
    # separable terms (Maxwellian factors of temperature 1 and vt)
    L = 2.0 * math.pi / k
    n_p = 9.0 / (10.0 * math.sqrt(2.0 * math.pi))
    n_b = 2.0 / (10.0 * math.sqrt(2.0 * math.pi))
    bulk = ("maxwell", {"c": n_p * math.sqrt(2.0 * math.pi)})
    beam = ("maxwell", {"u": u, "T": vt, "c": n_b * math.sqrt(2.0 * math.pi * vt)})
    one = ("const", {"c": 1.0})
    cs = ("cos", {"k": k, "c": alpha})
    terms = [[one, bulk], [one, beam], [cs, bulk], [cs, beam]]
    return Workload(name=f"bump_on_tail_1d1v_{N[0]}x{N[1]}", dx=1, dv=1, N=tuple(N),
                    lo=(0.0, -vmax), hi=(L, vmax), eps=eps, rank_cap=cap, dt=dt,
                    steps=steps, terms=terms, alpha=alpha, k=k)


def two_stream_1d1v(N=(64, 128), alpha=1e-3, k=0.2, v0=2.4, vmax=8.0, eps=1e-5, cap=16,
                    dt=0.1, steps=200) -> Workload:
    L = 2.0 * math.pi / k
    c = 1.0 / math.sqrt(2.0 * math.pi)
    terms = [[("const", {"c": 1.0}), ("two_stream", {"u": v0, "c": c})],
             [("cos", {"k": k, "c": alpha}), ("two_stream", {"u": v0, "c": c})]]
    return Workload(name=f"two_stream_1d1v_{N[0]}x{N[1]}", dx=1, dv=1, N=tuple(N),
                    lo=(0.0, -vmax), hi=(L, vmax), eps=eps, rank_cap=cap, dt=dt,
                    steps=steps, terms=terms, alpha=alpha, k=k)


def landau_2d2v(n=64, alpha=0.01, k=0.5, vmax=6.0, eps=1e-5, cap=32, dt=0.2,
                steps=200) -> Workload:
    L = 2.0 * math.pi / k
    mx = ("maxwell", {})
    one = ("const", {"c": 1.0})
    terms = [[one, one, mx, mx],
             [("cos", {"k": k, "c": alpha}), one, mx, mx],
             [one, ("cos", {"k": k, "c": alpha}), mx, mx]]
    return Workload(name=f"landau_2d2v_{n}^4", dx=2, dv=2, N=(n, n, n, n),
                    lo=(0.0, 0.0, -vmax, -vmax), hi=(L, L, vmax, vmax), eps=eps,
                    rank_cap=cap, dt=dt, steps=steps, terms=terms, alpha=alpha, k=k)


def two_stream_2d2v(n=128, alpha=0.005, k=0.2, v0=2.4, vmax=8.0, eps=5e-4, cap=48,
                    dt=0.1, steps=400) -> Workload:
    # f0 = (1 + a(cos k x1 + cos k x2)) / (4 pi) (e^{-(v1-v0)^2/2} + e^{-(v1+v0)^2/2}) e^{-v2^2/2}
    L = 2.0 * math.pi / k
    c = 1.0 / (4.0 * math.pi)
    ts = ("two_stream", {"u": v0, "c": c})
    g = ("maxwell", {"c": math.sqrt(2.0 * math.pi)})       # exp(-v^2/2)
    one = ("const", {"c": 1.0})
    terms = [[one, one, ts, g],
             [("cos", {"k": k, "c": alpha}), one, ts, g],
             [one, ("cos", {"k": k, "c": alpha}), ts, g]]
    return Workload(name=f"two_stream_2d2v_{n}^4", dx=2, dv=2, N=(n, n, n, n),
                    lo=(0.0, 0.0, -vmax, -vmax), hi=(L, L, vmax, vmax), eps=eps,
                    rank_cap=cap, dt=dt, steps=steps, terms=terms, alpha=alpha, k=k)


def bump_on_tail_2d2v(N=(128, 128, 128, 128), alpha=0.04, k=0.3, u=4.5, vt=2.4, vmax=13.0, eps=1e-4,
                      cap=48, dt=0.0625, steps=480) -> Workload:
    # f0 = (1 + alpha cos k x1 cos k x2) (n_p exp(-|v|^2/2) + n_b exp(-((v1-u)^2 + v2^2)/(2 vt))),
    # n_p = 17/(40 pi), n_b = 3/(40 pi vt), so that n_p 2 pi + n_b 2 pi vt = 1: total density 1
    # (the printed overall factor 1/(2 sqrt(2 pi))^2 would make it 1/(8 pi); reading: the
    # densities already carry the normalisation).  Four separable terms: (1, cos cos) x
    # (bulk, beam).  dt 0.0625: CFL 5 in x at v = 13 on 128 points.
    L = 2.0 * math.pi / k
    n_p = 17.0 / (40.0 * math.pi)
    n_b = 3.0 / (40.0 * math.pi * vt)
    b1 = ("maxwell", {"c": n_p * 2.0 * math.pi})            # n_p exp(-v1^2/2) (2 pi / sqrt(2 pi) each)
    b2 = ("maxwell", {})                                     # exp(-v2^2/2) / sqrt(2 pi)
    m1 = ("maxwell", {"u": u, "T": vt, "c": n_b * 2.0 * math.pi * vt})
    m2 = ("maxwell", {"T": vt})
    one = ("const", {"c": 1.0})
    ca = ("cos", {"k": k, "c": alpha})
    cb = ("cos", {"k": k, "c": 1.0})
    terms = [[one, one, b1, b2], [one, one, m1, m2], [ca, cb, b1, b2], [ca, cb, m1, m2]]
    N = tuple(N)
    return Workload(name=f"bump_on_tail_2d2v_{N[0]}x{N[1]}x{N[2]}x{N[3]}", dx=2, dv=2, N=N,
                    lo=(0.0, 0.0, -vmax, -vmax), hi=(L, L, vmax, vmax), eps=eps,
                    rank_cap=cap, dt=dt, steps=steps, terms=terms, alpha=alpha, k=k)


def ensemble(n_runs: int = 64, seed: int = 20261202, sizes=(32, 64, 128), cap_range=(8, 48),
             dt: float = 0.1) -> List[Workload]:
    """An ensemble of uneven runs: kinds cycle through 1D-1V Landau, 1D-1V two-stream,
    2D-2V Landau, 2D-2V two-stream; alpha ~ U[0.001, 0.5] (two-stream: alpha / 10),
    k ~ U[0.2, 0.6] (L = 2 pi / k per spatial dimension), points per dimension drawn from
    `sizes` (2D-2V: one size for all four dimensions), rank caps ~ U{cap_range}, eps 1e-5,
    dt 0.1.  Seeded numpy Generator (PCG64)."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_runs):
        kind = r % 4
        alpha = float(rng.uniform(0.001, 0.5))
        k = float(rng.uniform(0.2, 0.6))
        cap = int(rng.integers(cap_range[0], cap_range[1] + 1))
        if kind < 2:
            N = (int(rng.choice(sizes)), int(rng.choice(sizes)))
            w = (landau_1d1v(N=N, alpha=alpha, k=k, eps=1e-5, cap=cap, dt=dt) if kind == 0 else
                 two_stream_1d1v(N=N, alpha=alpha / 10, k=k, eps=1e-5, cap=cap, dt=dt))
        else:
            n = int(rng.choice(sizes))
            w = (landau_2d2v(n=n, alpha=alpha, k=k, eps=1e-5, cap=cap, dt=dt) if kind == 2 else
                 two_stream_2d2v(n=n, alpha=alpha / 10, k=k, eps=1e-5, cap=cap, dt=dt))
        w.name = f"run{r:02d}_{w.name}"
        out.append(w)
    return out


def workload_by_name(name: str) -> Workload:
    table = {
        "landau_1d1v": lambda: landau_1d1v(),
        "landau_2d2v": lambda: landau_2d2v(),
        "two_stream_2d2v": lambda: two_stream_2d2v(),
        "strong_landau_2d2v": lambda: landau_2d2v(n=128, alpha=0.5, cap=64, dt=0.2),
        "two_stream_1d1v": lambda: two_stream_1d1v(),
        "bump_on_tail_1d1v": lambda: bump_on_tail_1d1v(),
        "bump_on_tail_2d2v": lambda: bump_on_tail_2d2v(),
    }
    return table[name]()


# --------------------------------------------------------------------------------------
# Random inputs for parity tests (seeded).
# --------------------------------------------------------------------------------------

@dataclass
class RandomHT:
    """Raw random factors of a hierarchical-Tucker tensor for the trees
    d=2: root{0,1};  d=4: root{12{0,1}, 34{2,3}}.  Layouts: U[mu] is (N_mu, r_mu)
    row-major; B12 is (r0, r1, r12); B34 is (r2, r3, r34); Broot is (r_left, r_right)."""
    N: tuple
    U: list
    B12: Optional[np.ndarray]
    B34: Optional[np.ndarray]
    Broot: np.ndarray


def random_ht(N: Sequence[int], ranks: Sequence[int], seed: int, smooth: bool = True) -> RandomHT:
    """Seeded random HT factors.  ``ranks`` = leaf ranks (d of them) followed, for d=4, by
    (r12, r34).  With ``smooth`` the leaf columns are random trigonometric polynomials of
    low degree so that the tensor is a smooth periodic function (interpolation errors then
    stay small, like the paper's smooth distributions)."""
    rng = np.random.default_rng(seed)
    d = len(N)
    U = []
    for m in range(d):
        n, r = N[m], ranks[m]
        if smooth:
            t = 2.0 * math.pi * (np.arange(n) + 0.5) / n
            cols = []
            for _ in range(r):
                a = rng.standard_normal(4)
                b = rng.standard_normal(4)
                col = sum(a[q] * np.cos(q * t) + b[q] * np.sin(q * t) for q in range(4)) / 2.0
                cols.append(col)
            U.append(np.stack(cols, axis=1))
        else:
            U.append(rng.standard_normal((n, r)))
    if d == 2:
        Broot = rng.standard_normal((ranks[0], ranks[1])) / math.sqrt(ranks[0])
        return RandomHT(tuple(N), U, None, None, Broot)
    r12, r34 = ranks[4], ranks[5]
    B12 = rng.standard_normal((ranks[0], ranks[1], r12)) / math.sqrt(ranks[0] * ranks[1])
    B34 = rng.standard_normal((ranks[2], ranks[3], r34)) / math.sqrt(ranks[2] * ranks[3])
    Broot = rng.standard_normal((r12, r34)) / math.sqrt(r12)
    return RandomHT(tuple(N), U, B12, B34, Broot)


def random_tuples(N: Sequence[int], n: int, seed: int) -> np.ndarray:
    """n uniformly random grid index tuples, int32[n][d]."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, N[m], size=n) for m in range(len(N))], axis=1).astype(np.int32)


def random_field(Nx: Sequence[int], dx: int, amplitude: float, seed: int) -> np.ndarray:
    """A smooth random periodic vector field E, float64[dx][prod Nx] (row-major, x1 slowest)."""
    rng = np.random.default_rng(seed)
    grids = [2.0 * math.pi * (np.arange(n) + 0.5) / n for n in Nx]
    mesh = np.meshgrid(*grids, indexing="ij")
    out = []
    for _ in range(dx):
        f = np.zeros(mesh[0].shape)
        for _ in range(3):
            kk = rng.integers(0, 3, size=dx)
            ph = rng.uniform(0, 2 * math.pi)
            arg = sum(kk[m] * mesh[m] for m in range(dx)) + ph
            f += rng.standard_normal() * np.cos(arg)
        out.append(amplitude * f.reshape(-1))
    return np.stack(out)
