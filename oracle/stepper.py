"""SLAR, SLAR_VP (third-order commutator-free RK exponential integrator) and the
LoMaC-coupled time step of the flowchart (Sec. 3.1, Eq. slarvp; Sec. 3.2.3 and the
flowchart figure; Sec. 4 start-up with DIRK3 then BDF3).

Test infrastructure: part of the FP64 oracle, never called by the CUDA path.

Readings:
* RKEI = CF3 of Celledoni, Marthinsen and Owren (2003):
    Y2 = exp(dt/3 F(Y1)) Y1,  Y3 = exp(2dt/3 F(Y2)) Y1,
    Y^{n+1} = exp(dt(-F(Y1)/12 + 3F(Y3)/4)) Y2,
  with F(Y) the frozen-field advection operator of the field of Y.  The combination in
  the last exponential is itself a frozen-field advection over tau = 2dt/3 with the field
  E_c = -E1/8 + 9E3/8 (the advection operator is linear in v-speed and field).
* Each exponential is one SLAR call (cross approximation of the SL-updated tensor,
  then HSVD truncation).
* The LoMaC state F^{n+1} = HT(F*) + separable correction is never truncated; the next
  SLAR samples its entries (interpolation is linear, so both parts are interpolated with
  the same weights).
* Time stepping of the macroscopic system: DIRK3 (each stage: one SLAR_VP to the stage
  time c_i dt from F^n, one JFNK) for the first two steps, variable-step BDF3 afterwards.
  Without LoMaC the step is F^{n+1} = F*.  The DIRK-only coupling (the first of the two
  high-order options of Sec. 3.2.3) takes the DIRK3 step every time: three SLAR_VP calls
  and three JFNK solves per step instead of one of each.
"""
from __future__ import annotations

from dataclasses import dataclass, field as dfield
from typing import List, Optional

import numpy as np

from . import cross, field, lomac, macro, net, precond, sl
from .ht import HT, from_terms, truncate
from .sl import PhaseGrid


@dataclass
class Params:
    eps: float
    cap: int
    newton_tol: float = 1e-12
    krylov_tol: float = 1e-4
    krylov_restart: int = 30
    newton_max: int = 20
    krylov_max: int = 200
    foot: str = "rk3"
    delta: float = lomac.DELTA_DEFAULT
    lomac: bool = True
    # Newton-Krylov solve of the BDF3 steps: "none" (the paper's plain JFNK), "circulant"
    # (block-circulant right preconditioner) or "learned" (network guess and block on top
    # of the circulant preconditioner; plain JFNK from U* is the fallback).
    precond: str = "none"
    net_theta: Optional[np.ndarray] = None
    net_hidden: int = net.HIDDEN
    probes: int = 4
    # fibres per cross-approximation step (1: classical partial pivoting; > 1: block cross)
    block: int = 1
    # DIRK3 every step (the DIRK coupling of Sec. 3.2.3) instead of BDF3 after the start-up
    dirk_only: bool = False


@dataclass
class State:
    F: HT
    U: np.ndarray                      # conserved variables (dv+2, Nx)
    hist: List[np.ndarray]             # previous U (most recent first), for BDF3
    n_i: float
    dts: List[float] = dfield(default_factory=list)   # previous step sizes, most recent first
    t: float = 0.0
    step: int = 0


@dataclass
class StepStats:
    entries: int = 0
    ranks: list = dfield(default_factory=list)
    newton: int = 0
    krylov: int = 0
    residual: float = 0.0
    converged: bool = True
    W: float = 0.0
    aca_ranks: list = dfield(default_factory=list)
    guess_used: bool = False
    fallback: bool = False
    pivots: list = dfield(default_factory=list)   # (row, column) pivots of each SLAR call


def init_state(factors, g: PhaseGrid, prm: Params) -> State:
    """F^0 = HSVD-truncated HT of the separable initial data; n_i = mean M0(F^0);
    U^0 = U(F^0)."""
    F0 = truncate(from_terms(factors), prm.eps, prm.cap)
    mom = field.moments(F0, g)
    n_i = float(np.mean(mom[0]))
    U0 = lomac.conserved_from_moments(mom, g, n_i)
    return State(F=F0, U=U0, hist=[], n_i=n_i)


def field_of(F: HT, g: PhaseGrid, n_i: float) -> np.ndarray:
    """E of a state: rho = n_i - M0(F), spectral Poisson, E = -grad phi."""
    M0 = field.ht_moment(F, g, field.moment_monomials(g.dv)[0])
    if F.corr is not None:
        M0 = M0 + field.correction_moment(F.corr, g, field.moment_monomials(g.dv)[0])
    return field.poisson_field(n_i - M0, g)[1]


def slar(F: HT, E: np.ndarray, tau: float, g: PhaseGrid, prm: Params, pivots=None):
    """SLAR(F; E, tau, eps): cross approximation of the SL-updated tensor, then truncation."""
    fn = lambda idx: sl.sl_eval(F, E, tau, idx, g, prm.foot)
    return cross.htaca(fn, g.N, prm.eps, prm.cap, pivots=pivots, return_info=True, block=prm.block)


def slar_vp(F: HT, dt: float, g: PhaseGrid, prm: Params, n_i: float, pivots=None):
    """One SLAR_VP step (Eq. slarvp) by CF3.  Returns (F*, info)."""
    piv = pivots or [None, None, None]
    E1 = field_of(F, g, n_i)
    Y2, i1 = slar(F, E1, dt / 3.0, g, prm, piv[0])
    E2 = field_of(Y2, g, n_i)
    Y3, i2 = slar(F, E2, 2.0 * dt / 3.0, g, prm, piv[1])
    E3 = field_of(Y3, g, n_i)
    Ec = -E1 / 8.0 + 9.0 * E3 / 8.0
    Fs, i3 = slar(Y2, Ec, 2.0 * dt / 3.0, g, prm, piv[2])
    info = dict(entries=i1["entries"] + i2["entries"] + i3["entries"],
                pivots=[i1["pivots"], i2["pivots"], i3["pivots"]],
                ranks=i3["ranks"], fields=(E1, E2, E3),
                aca_ranks=[i1["aca_rank"], i2["aca_rank"], i3["aca_rank"]])
    return Fs, info


def _solve(cl: macro.Closure, rhs: np.ndarray, coef: float, U_guess: np.ndarray, tol_abs: float,
           prm: Params):
    """JFNK on G(U) = U - rhs - coef K(U) = 0."""
    Gfun = lambda U: U - rhs - coef * macro.K_operator(U, cl)
    return macro.jfnk(Gfun, U_guess, tol_abs, prm.krylov_tol, prm.krylov_restart,
                      prm.newton_max, prm.krylov_max)


def spatial_shape(g: PhaseGrid):
    """The spatial grid as a 2D array shape (n0, n1), n1 = 1 in one dimension."""
    return (g.N[0], g.N[1]) if g.dx == 2 else (g.N[0], 1)


def _solve_precond(Gfun, Un_prev: np.ndarray, Ustar: np.ndarray, tol_abs: float, prm: Params,
                   shape2d, stats: StepStats):
    """Preconditioned (and, with a network, warm-started) JFNK; plain JFNK from U* if it
    does not converge."""
    m = Ustar.shape[0]
    U0, y = Ustar, None
    if prm.precond == "learned":
        x, sD = net.features(Un_prev, Ustar, shape2d)
        y, _ = net.forward(prm.net_theta, x, m, prm.net_hidden)
        Ug = net.guess_from_output(y, Ustar, sD)
        if np.max(np.abs(Gfun(Ug))) <= np.max(np.abs(Gfun(Ustar))):
            U0 = Ug
            stats.guess_used = True
    P = precond.circulant_blocks(Gfun, U0, Gfun(U0), shape2d)
    if y is None:
        Papply = lambda v: precond.apply_circulant(P, v)
    else:
        Papply = lambda v: precond.apply_circulant(P, net.apply_block(y, v))
    Un, ns = precond.jfnk_right(Gfun, U0, tol_abs, prm.krylov_tol, Papply, prm.krylov_restart,
                                prm.newton_max, prm.krylov_max)
    stats.newton, stats.krylov = ns.newton, ns.krylov
    stats.residual, stats.converged = ns.residual, ns.converged
    if not ns.converged:
        stats.fallback = True
        Un, ps = macro.jfnk(Gfun, Ustar, tol_abs, prm.krylov_tol, prm.krylov_restart,
                            prm.newton_max, prm.krylov_max)
        stats.newton += ps.newton
        stats.krylov += ps.krylov
        stats.residual, stats.converged = ps.residual, ps.converged
    return Un


def training_sample(Gfun, Un_prev: np.ndarray, Ustar: np.ndarray, Unew: np.ndarray, shape2d,
                    probes: np.ndarray) -> net.Sample:
    """Training sample of one BDF3 solve: features, scaled guess target, and probe pairs
    (v_s, J P v_s) with J and the block-circulant P at U*.  probes (S-1, m, NX) are the
    random directions; the first direction is the residual -G(U*), RMS-scaled per channel."""
    m = Ustar.shape[0]
    x, sD = net.features(Un_prev, Ustar, shape2d)
    t = ((Unew - Ustar) / sD[:, None]).reshape((m,) + tuple(shape2d))
    G0 = Gfun(Ustar)
    P = precond.circulant_blocks(Gfun, Ustar, G0, shape2d)
    v0 = -G0 / net.rms_scales(G0, net.SCALE_FLOOR)[:, None]
    vs = [v0] + [p for p in probes]
    ws = [precond.fd_jv(Gfun, Ustar, G0, precond.apply_circulant(P, v)) for v in vs]
    shp = (len(vs), m) + tuple(shape2d)
    return net.Sample(x=x, t=t, v=np.stack(vs).reshape(shp), w=np.stack(ws).reshape(shp))


def sl_step(st: State, dt: float, g: PhaseGrid, prm: Params, pivots=None,
            record: Optional[list] = None, probes: Optional[np.ndarray] = None) -> StepStats:
    """Advance the state by one step (flowchart of Sec. 3.2.3)."""
    stats = StepStats()
    if not prm.lomac:
        Fs, info = slar_vp(st.F, dt, g, prm, st.n_i, pivots)
        st.F = Fs
        st.U = lomac.conserved_from_moments(field.moments(Fs, g), g, st.n_i)
        stats.entries, stats.ranks = info["entries"], info["ranks"]
        stats.aca_ranks = info["aca_ranks"]
        stats.pivots = info["pivots"]
    elif st.step < 2 or prm.dirk_only:
        A, c = macro.dirk3_tableau()
        tol_abs = macro.newton_tol_abs(prm.newton_tol, st.U)
        Ks = []
        for i in range(3):
            Fs, info = slar_vp(st.F, c[i] * dt, g, prm, st.n_i, None if pivots is None else pivots[i])
            stats.entries += info["entries"]
            stats.aca_ranks += info["aca_ranks"]
            stats.pivots += info["pivots"]
            cl = macro.make_closure(Fs, g, st.n_i, prm.delta)
            rhs = st.U + dt * sum(A[i, j] * Ks[j] for j in range(i)) if i else st.U.copy()
            Ustar = lomac.conserved_from_moments(cl.mom_star, g, st.n_i)
            Ui, ns = _solve(cl, rhs, dt * A[i, i], Ustar, tol_abs, prm)
            stats.newton += ns.newton
            stats.krylov += ns.krylov
            stats.residual = max(stats.residual, ns.residual)
            stats.converged &= ns.converged
            Ks.append(macro.K_operator(Ui, cl))
        # stiffly accurate: U^{n+1} = U_3 with the stage-3 closure
        st.hist = [st.U] + st.hist[:1]
        st.U = Ui
        st.F = lomac.correct(Fs, cl.basis, Ui, g, st.n_i)
        stats.ranks = info["ranks"]
    else:
        Fs, info = slar_vp(st.F, dt, g, prm, st.n_i, pivots)
        stats.entries, stats.ranks = info["entries"], info["ranks"]
        stats.aca_ranks = info["aca_ranks"]
        stats.pivots = info["pivots"]
        cl = macro.make_closure(Fs, g, st.n_i, prm.delta)
        # variable-step BDF3 (equal steps: the fixed-step table)
        a, beta = macro.bdf3_variable((dt, st.dts[0], st.dts[1]))
        rhs = a[0] * st.U + a[1] * st.hist[0] + a[2] * st.hist[1]
        tol_abs = macro.newton_tol_abs(prm.newton_tol, st.U)
        Ustar = lomac.conserved_from_moments(cl.mom_star, g, st.n_i)
        coef = beta * dt
        Gfun = lambda U: U - rhs - coef * macro.K_operator(U, cl)
        if prm.precond == "none":
            Un, ns = _solve(cl, rhs, coef, Ustar, tol_abs, prm)
            stats.newton, stats.krylov = ns.newton, ns.krylov
            stats.residual, stats.converged = ns.residual, ns.converged
        else:
            Un = _solve_precond(Gfun, st.U, Ustar, tol_abs, prm, spatial_shape(g), stats)
        if record is not None:
            record.append(training_sample(Gfun, st.U, Ustar, Un, spatial_shape(g), probes))
        st.hist = [st.U] + st.hist[:1]
        st.U = Un
        st.F = lomac.correct(Fs, cl.basis, Un, g, st.n_i)
    st.t += dt
    st.step += 1
    st.dts = [dt] + st.dts[:1]
    stats.W = field.poisson_field(st.n_i - st.U[0], g)[2]
    return stats


def cfl_dt(st: State, g: PhaseGrid, cfl: float, dt_max: float,
           ratio_max: float = macro.BDF3_RATIO_MAX) -> float:
    """Adaptive step size (Sec. 3.2.3 adaptive time stepping; the dimension-wise CFL numbers
    lambda_i = a_i dt / Delta_i of Appendix A): dt = cfl / max_i(a_i / Delta_i) with the
    advection speeds a = max |v_m| in x_m and max |E_m| of the state's field in v_m, capped
    at dt_max and, after the start-up steps, at ratio_max times the previous step."""
    E = field_of(st.F, g, st.n_i)
    rate = 0.0
    for m in range(g.dx):
        vmax = float(np.max(np.abs(g.centres(g.dx + m))))
        rate = max(rate, vmax / g.h(m), float(np.max(np.abs(E[m]))) / g.h(g.dx + m))
    dt = dt_max if rate == 0.0 else min(dt_max, cfl / rate)
    if st.step >= 2 and st.dts:
        dt = min(dt, ratio_max * st.dts[0])
    return dt


def totals(st: State, g: PhaseGrid):
    """Total mass, momentum (per direction) and energy of the conserved variables."""
    cell = float(np.prod([g.h(m) for m in range(g.dx)]))
    return st.U.sum(axis=1) * cell
