"""Thin ctypes binding of libslar.so (include/slar.h).  Argument marshalling only: every
step of the method runs in the library's CUDA kernels.  Device arrays are torch CUDA
tensors (float64 / int32, contiguous); host arrays are numpy.

The library must have been built (``python -m paper_2606_29027_b300.build``); importing
this module without it raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libslar.so")

SLAR_OK, SLAR_EINVAL, SLAR_ENOMEM, SLAR_ECUDA, SLAR_ENOCONV, SLAR_ETIMEOUT, SLAR_ERANK, SLAR_ENAN = range(8)
SLAR_FP64, SLAR_FP32, SLAR_FP32_BF16X3, SLAR_FP32_BF16X6 = 0, 1, 2, 3
SLAR_LOMAC, SLAR_FOOT_EULER, SLAR_PROFILE, SLAR_PROFILE_EVAL = 1, 2, 4, 8
SLAR_PRECOND, SLAR_LEARNED, SLAR_NO_AUTOTUNE, SLAR_OWN_STREAM = 16, 32, 64, 128
SLAR_DIRK_ONLY = 256

# every entry point declared in include/slar.h
EXPORTED = ["slar_create", "slar_destroy", "slar_last_error", "init_ht", "sl_step", "ht_truncate",
            "moments", "lomac_correct", "poisson_field", "ht_eval", "sl_eval", "slar_advect",
            "slar_set_pivot_replay", "ht_export", "ht_import", "slar_get_conserved",
            "slar_set_conserved", "slar_sizes", "slar_launch_count", "slar_poisson_field_static",
            "slar_net_param_count", "slar_sample_floats", "slar_net_create", "slar_net_destroy",
            "slar_net_set_params", "slar_net_get_params", "slar_net_forward", "slar_net_loss_grad",
            "slar_net_train_step", "slar_attach_net", "slar_set_record", "slar_fma_peak",
            "slar_ensemble_step", "slar_stream", "slar_wait_probe", "slar_checkpoint",
            "slar_restore", "slar_cfl_dt"]
SLAR_MOM_M0, SLAR_MOM_M1, SLAR_MOM_M2, SLAR_MOM_FLUX, SLAR_MOM_ALL = 1, 2, 4, 8, 15


class Config(C.Structure):
    _fields_ = [("dx", C.c_int), ("dv", C.c_int), ("N", C.c_int * 4), ("lo", C.c_double * 4),
                ("hi", C.c_double * 4), ("eps", C.c_double), ("rank_cap", C.c_int),
                ("newton_tol", C.c_double), ("krylov_tol", C.c_double), ("krylov_restart", C.c_int),
                ("newton_max", C.c_int), ("krylov_max", C.c_int), ("precision", C.c_int),
                ("flags", C.c_int), ("delta_floor", C.c_double), ("aca_block", C.c_int),
                ("interp_order", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("entries", C.c_longlong), ("ranks", C.c_int * 6), ("aca_rank", C.c_int * 9),
                ("n_slar", C.c_int), ("newton", C.c_int), ("krylov", C.c_int),
                ("residual", C.c_double), ("converged", C.c_int), ("field_energy", C.c_double),
                ("totals", C.c_double * 4), ("eval_ms", C.c_double), ("eval_flop", C.c_double),
                ("launches", C.c_longlong), ("phase_ms", C.c_double * 6),
                ("guess_used", C.c_int), ("fallback", C.c_int), ("recorded", C.c_int),
                ("g_evals", C.c_int), ("eval_tile", C.c_int), ("rank_capped", C.c_int),
                ("pc_built", C.c_int)]

    def to_dict(self):
        return dict(entries=self.entries, ranks=list(self.ranks), aca_rank=list(self.aca_rank[: self.n_slar]),
                    newton=self.newton, krylov=self.krylov, residual=self.residual,
                    converged=bool(self.converged), field_energy=self.field_energy,
                    totals=list(self.totals), eval_ms=self.eval_ms, eval_flop=self.eval_flop,
                    launches=self.launches, phase_ms=list(self.phase_ms),
                    guess_used=bool(self.guess_used), fallback=bool(self.fallback),
                    recorded=bool(self.recorded), g_evals=self.g_evals, eval_tile=self.eval_tile,
                    rank_capped=self.rank_capped, pc_built=bool(self.pc_built))


class HTView(C.Structure):
    _fields_ = [("d", C.c_int), ("N", C.c_int * 4), ("rank", C.c_int * 6),
                ("U", C.POINTER(C.c_double) * 4), ("B12", C.POINTER(C.c_double)),
                ("B34", C.POINTER(C.c_double)), ("Broot", C.POINTER(C.c_double)),
                ("has_corr", C.c_int), ("dC", C.POINTER(C.c_double)), ("qv", C.POINTER(C.c_double))]


_lib = None


def load():
    """Load libslar.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} not built; run python -m paper_2606_29027_b300.build")
    lib = C.CDLL(LIB_PATH)
    P, I, D, LL = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    sig = {
        "slar_create": ([C.POINTER(Config), P, C.POINTER(P)], I),
        "slar_destroy": ([P], I),
        "slar_last_error": ([P], C.c_char_p),
        "init_ht": ([P, I, P], I),
        "sl_step": ([P, D, C.POINTER(Stats)], I),
        "ht_truncate": ([P, D, I], I),
        "moments": ([P, C.c_uint, P], I),
        "lomac_correct": ([P, P], I),
        "poisson_field": ([P, P, P, P, C.POINTER(D)], I),
        "ht_eval": ([P, LL, P, P], I),
        "sl_eval": ([P, D, P, LL, P, P], I),
        "slar_advect": ([P, D, P, C.POINTER(I), C.POINTER(LL)], I),
        "slar_set_pivot_replay": ([P, I, I, P], I),
        "ht_export": ([P, C.POINTER(HTView)], I),
        "ht_import": ([P, C.POINTER(HTView)], I),
        "slar_get_conserved": ([P, P, C.POINTER(D)], I),
        "slar_set_conserved": ([P, P, D], I),
        "slar_sizes": ([P, C.POINTER(I), C.POINTER(I)], I),
        "slar_launch_count": ([C.POINTER(LL)], I),
        "slar_poisson_field_static": ([I, P, P, P, P, P, C.POINTER(D), P], I),
        "slar_net_param_count": ([I, I, C.POINTER(LL)], I),
        "slar_sample_floats": ([I, I, I, C.POINTER(LL)], I),
        "slar_net_create": ([I, I, I, I, I, P, C.POINTER(P)], I),
        "slar_net_destroy": ([P], I),
        "slar_net_set_params": ([P, P, LL], I),
        "slar_net_get_params": ([P, P, LL], I),
        "slar_net_forward": ([P, P, I, P], I),
        "slar_net_loss_grad": ([P, P, I, P, I, C.POINTER(D), P], I),
        "slar_net_train_step": ([P, P, I, P, I, C.c_float, C.POINTER(D)], I),
        "slar_attach_net": ([P, P], I),
        "slar_set_record": ([P, P, I, C.c_ulonglong], I),
        "slar_fma_peak": ([I, I, C.POINTER(D), P], I),
        "slar_ensemble_step": ([P, I, P, I, P], I),
        "slar_stream": ([P, C.POINTER(P)], I),
        "slar_wait_probe": ([LL, P, P], I),
        "slar_checkpoint": ([P, C.c_char_p], I),
        "slar_restore": ([P, C.c_char_p], I),
        "slar_cfl_dt": ([P, D, D, C.POINTER(D)], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    n = C.c_longlong()
    st = load().slar_launch_count(C.byref(n))
    if st != SLAR_OK:
        raise SlarError(st, "slar_launch_count failed")
    return n.value


def poisson_field_static(N, L, rho, E, phi=None, stream=None, energy=True):
    """Context-free, allocation-free spectral Poisson solve (see include/slar.h).  rho, E,
    phi: torch CUDA float64 tensors.  Returns the electric energy (or None)."""
    import torch
    dx = len(N)
    Na = (C.c_int * 2)(*[int(n) for n in N] + [1] * (2 - dx))
    La = (C.c_double * 2)(*[float(x) for x in L] + [1.0] * (2 - dx))
    W = C.c_double()
    st = stream if stream is not None else torch.cuda.current_stream()
    status = load().slar_poisson_field_static(dx, Na, La, C.c_void_p(_ptr(rho)), C.c_void_p(_ptr(E)),
                                              C.c_void_p(_ptr(phi)), C.byref(W) if energy else None,
                                              C.c_void_p(st.cuda_stream))
    if status != SLAR_OK:
        raise SlarError(status, "slar_poisson_field_static failed")
    return W.value if energy else None


def wait_probe(polls: int, status, stream=None) -> int:
    """Run the bounded-wait probe (see include/slar.h); returns the status code
    (SLAR_ETIMEOUT when the wait gave up).  status: a CUDA int32 tensor of one element."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    return load().slar_wait_probe(int(polls), C.c_void_p(_ptr(status)), C.c_void_p(st.cuda_stream))


def fma_peak(fp64: bool, iters: int = 0, stream=None) -> float:
    """Measured FMA throughput of the GPU in TFLOP/s (see include/slar.h)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    it = iters or (512 if fp64 else 4096)
    t = C.c_double()
    status = load().slar_fma_peak(1 if fp64 else 0, it, C.byref(t), C.c_void_p(st.cuda_stream))
    if status != SLAR_OK:
        raise SlarError(status, "slar_fma_peak failed")
    return t.value


class SlarError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"slar status {status}: {msg}")
        self.status = status


def _ptr(t) -> int:
    """Device pointer of a contiguous torch tensor (0 for None)."""
    if t is None:
        return 0
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_config(workload=None, *, dx=None, dv=None, N=None, lo=None, hi=None, eps=1e-6, rank_cap=16,
                newton_tol=1e-12, krylov_tol=1e-4, krylov_restart=30, newton_max=20, krylov_max=200,
                precision="fp64", lomac=True, foot="rk3", delta_floor=1e-12, profile=False,
                profile_eval=False, solver="plain", autotune=True, own_stream=False,
                aca_block=1, dirk_only=False, interp_order=2) -> Config:
    """solver: "plain" (the paper's JFNK), "precond" (block-circulant preconditioner) or
    "learned" (network warm start; attach a network with Context.attach_net)."""
    if workload is not None:
        dx, dv, N, lo, hi = workload.dx, workload.dv, workload.N, workload.lo, workload.hi
        eps, rank_cap = workload.eps, workload.rank_cap
        newton_tol, krylov_tol, lomac = workload.newton_tol, workload.krylov_tol, workload.lomac
    cfg = Config()
    cfg.dx, cfg.dv = dx, dv
    d = dx + dv
    for m in range(4):
        cfg.N[m] = int(N[m]) if m < d else 1
        cfg.lo[m] = float(lo[m]) if m < d else 0.0
        cfg.hi[m] = float(hi[m]) if m < d else 1.0
    cfg.eps, cfg.rank_cap = eps, rank_cap
    cfg.newton_tol, cfg.krylov_tol = newton_tol, krylov_tol
    cfg.krylov_restart, cfg.newton_max, cfg.krylov_max = krylov_restart, newton_max, krylov_max
    cfg.precision = {"fp64": SLAR_FP64, "fp32": SLAR_FP32, "bf16x3": SLAR_FP32_BF16X3,
                     "bf16x6": SLAR_FP32_BF16X6}[precision]
    cfg.flags = ((SLAR_LOMAC if lomac else 0) | (SLAR_FOOT_EULER if foot == "euler" else 0)
                 | (SLAR_PROFILE if profile else 0) | (SLAR_PROFILE_EVAL if profile_eval else 0)
                 | {"plain": 0, "precond": SLAR_PRECOND, "learned": SLAR_LEARNED}[solver]
                 | (0 if autotune else SLAR_NO_AUTOTUNE) | (SLAR_OWN_STREAM if own_stream else 0)
                 | (SLAR_DIRK_ONLY if dirk_only else 0))
    cfg.delta_floor = delta_floor
    cfg.aca_block = int(aca_block)
    cfg.interp_order = int(interp_order)
    return cfg


class Context:
    """One library context bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, cfg: Config, stream=None):
        import torch
        self.lib = load()
        self.cfg = cfg
        self.d = cfg.dx + cfg.dv
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        st = self.lib.slar_create(C.byref(cfg), C.c_void_p(stream.cuda_stream), C.byref(h))
        if st != SLAR_OK:
            raise SlarError(st, "slar_create failed")
        self.h = h
        if cfg.flags & SLAR_OWN_STREAM:
            sp = C.c_void_p()
            self.lib.slar_stream(self.h, C.byref(sp))
            self.stream = torch.cuda.ExternalStream(sp.value)
        nm, nx = C.c_int(), C.c_int()
        self.lib.slar_sizes(self.h, C.byref(nm), C.byref(nx))
        self.n_mom, self.NX = nm.value, nx.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.slar_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        """Raise on an error status.  SLAR_ERANK is a warning (the call completed and its
        result is valid): it is kept in self.last_status instead."""
        self.last_status = st
        if st not in (SLAR_OK, SLAR_ERANK):
            raise SlarError(st, self.lib.slar_last_error(self.h).decode())

    # ---- entry points ----
    def init_ht(self, factors):
        """factors: [term][mu] -> 1D numpy arrays."""
        T = len(factors)
        flat = np.concatenate([np.concatenate([np.asarray(f, np.float64) for f in term]) for term in factors])
        flat = np.ascontiguousarray(flat)
        self._check(self.lib.init_ht(self.h, T, flat.ctypes.data_as(C.c_void_p)))

    def step(self, dt: float) -> Stats:
        st = Stats()
        status = self.lib.sl_step(self.h, dt, C.byref(st))
        if status not in (SLAR_OK, SLAR_ENOCONV, SLAR_ERANK):
            self._check(status)
        self.last_status = status
        st.status = status
        return st

    def truncate(self, eps: float, cap: int):
        self._check(self.lib.ht_truncate(self.h, eps, cap))

    def moments(self, out, mask: int = 0):
        """Moments selected by `mask` (SLAR_MOM_*; 0 = all) into out [n_sel][NX]."""
        self._check(self.lib.moments(self.h, int(mask), C.c_void_p(_ptr(out))))

    def checkpoint(self, path: str):
        self._check(self.lib.slar_checkpoint(self.h, os.fsencode(path)))

    def restore(self, path: str):
        self._check(self.lib.slar_restore(self.h, os.fsencode(path)))

    def cfl_dt(self, cfl: float, dt_max: float) -> float:
        """Step size of the adaptive rule (see include/slar.h, slar_cfl_dt)."""
        dt = C.c_double()
        self._check(self.lib.slar_cfl_dt(self.h, float(cfl), float(dt_max), C.byref(dt)))
        return dt.value

    def lomac_correct(self, U_target):
        self._check(self.lib.lomac_correct(self.h, C.c_void_p(_ptr(U_target))))

    def poisson_field(self, rho, E, phi=None) -> float:
        W = C.c_double()
        self._check(self.lib.poisson_field(self.h, C.c_void_p(_ptr(rho)), C.c_void_p(_ptr(E)),
                                           C.c_void_p(_ptr(phi)), C.byref(W)))
        return W.value

    def ht_eval(self, idx, out):
        self._check(self.lib.ht_eval(self.h, idx.shape[0], C.c_void_p(_ptr(idx)), C.c_void_p(_ptr(out))))

    def sl_eval(self, tau, E, idx, out):
        self._check(self.lib.sl_eval(self.h, tau, C.c_void_p(_ptr(E)), idx.shape[0],
                                     C.c_void_p(_ptr(idx)), C.c_void_p(_ptr(out))))

    def advect(self, tau, E):
        k, n = C.c_int(), C.c_longlong()
        self._check(self.lib.slar_advect(self.h, tau, C.c_void_p(_ptr(E)), C.byref(k), C.byref(n)))
        return k.value, n.value

    def set_pivot_replay(self, calls):
        """calls: list (per SLAR call) of lists of (i, j) pivots."""
        if not calls:
            self._check(self.lib.slar_set_pivot_replay(self.h, 0, 1, None))
            return
        kmax = max(len(c) for c in calls) + 1
        arr = -np.ones((len(calls), kmax, 2), dtype=np.int32)
        for a, piv in enumerate(calls):
            for k, (i, j) in enumerate(piv):
                arr[a, k] = (i, j)
        arr = np.ascontiguousarray(arr)
        self._check(self.lib.slar_set_pivot_replay(self.h, len(calls), kmax, arr.ctypes.data_as(C.c_void_p)))

    def attach_net(self, net: Optional["Net"]):
        """Use `net` for the SLAR_LEARNED warm start (None detaches)."""
        self._net = net
        self._check(self.lib.slar_attach_net(self.h, net.h if net is not None else None))

    def set_record(self, sample, n_probes: int, seed: int):
        """Write the training sample of the next BDF3 step into `sample` (torch CUDA float32
        tensor of sample_floats(dv+2, NX, n_probes) elements; None cancels)."""
        if sample is not None and (sample.numel() != sample_floats(self.cfg.dv + 2, self.NX, n_probes)
                                   or sample.dtype.itemsize != 4):
            raise ValueError("sample buffer has the wrong size or type")
        self._rec = sample
        self._check(self.lib.slar_set_record(self.h, C.c_void_p(_ptr(sample)), int(n_probes),
                                             C.c_ulonglong(seed)))

    def get_conserved(self, U_out):
        ni = C.c_double()
        self._check(self.lib.slar_get_conserved(self.h, C.c_void_p(_ptr(U_out)), C.byref(ni)))
        return ni.value

    def set_conserved(self, U, n_i):
        self._check(self.lib.slar_set_conserved(self.h, C.c_void_p(_ptr(U)), float(n_i)))

    def export(self) -> dict:
        """Copy the HT state to host: dict(U=[...], B12, B34, Broot, dC, qv) in the library
        layouts ([p][a][b] transfer tensors)."""
        v = HTView()
        self._check(self.lib.ht_export(self.h, C.byref(v)))
        d = v.d
        r = list(v.rank)
        N = list(v.N)
        out = dict(d=d, ranks=r, N=N, has_corr=bool(v.has_corr))
        U = [np.zeros((N[m], r[m])) for m in range(d)]
        for m in range(d):
            v.U[m] = _dptr(U[m])
        if d == 4:
            B12 = np.zeros((r[4], r[0], r[1]))
            B34 = np.zeros((r[5], r[2], r[3]))
            Broot = np.zeros((r[4], r[5]))
            v.B12, v.B34 = _dptr(B12), _dptr(B34)
        else:
            B12 = B34 = None
            Broot = np.zeros((r[0], r[1]))
        v.Broot = _dptr(Broot)
        dv = self.cfg.dv
        dC = np.zeros((dv + 2, self.NX))
        qv = np.zeros((3, dv, N[self.cfg.dx]))
        v.dC, v.qv = _dptr(dC), _dptr(qv)
        self._check(self.lib.ht_export(self.h, C.byref(v)))
        out.update(U=U, B12=B12, B34=B34, Broot=Broot)
        if out["has_corr"]:
            out.update(dC=dC, qv=qv)
        return out

    def import_ht(self, U, Broot, B12=None, B34=None, dC=None, qv=None):
        """Set the state from host arrays in the library layouts."""
        v = HTView()
        v.d = self.d
        keep = []
        for m in range(self.d):
            u = np.ascontiguousarray(U[m], dtype=np.float64)
            keep.append(u)
            v.N[m] = u.shape[0]
            v.rank[m] = u.shape[1]
            v.U[m] = _dptr(u)
        br = np.ascontiguousarray(Broot, dtype=np.float64)
        keep.append(br)
        v.Broot = _dptr(br)
        if self.d == 4:
            b12 = np.ascontiguousarray(B12, dtype=np.float64)
            b34 = np.ascontiguousarray(B34, dtype=np.float64)
            keep += [b12, b34]
            v.B12, v.B34 = _dptr(b12), _dptr(b34)
            v.rank[4], v.rank[5] = b12.shape[0], b34.shape[0]
        if dC is not None:
            dc = np.ascontiguousarray(dC, dtype=np.float64)
            q = np.ascontiguousarray(qv, dtype=np.float64)
            keep += [dc, q]
            v.has_corr = 1
            v.dC, v.qv = _dptr(dc), _dptr(q)
        self._check(self.lib.ht_import(self.h, C.byref(v)))


def ensemble_step(contexts, dts, threads: int = 16):
    """Advance every context by one step concurrently (slar_ensemble_step); the contexts must
    have distinct streams.  Returns the list of Stats."""
    n = len(contexts)
    arr = (C.c_void_p * n)(*[c.h.value for c in contexts])
    d = (C.c_double * n)(*[float(x) for x in dts])
    stats = (Stats * n)()
    status = load().slar_ensemble_step(arr, n, d, int(threads), stats)
    if status not in (SLAR_OK, SLAR_ENOCONV, SLAR_ERANK):
        raise SlarError(status, "slar_ensemble_step failed")
    return list(stats)


def net_param_count(m: int, hidden: int = 32) -> int:
    n = C.c_longlong()
    st = load().slar_net_param_count(m, hidden, C.byref(n))
    if st != SLAR_OK:
        raise SlarError(st, "slar_net_param_count failed")
    return n.value


def sample_floats(m: int, nx: int, n_probes: int) -> int:
    n = C.c_longlong()
    st = load().slar_sample_floats(m, nx, n_probes, C.byref(n))
    if st != SLAR_OK:
        raise SlarError(st, "slar_sample_floats failed")
    return n.value


class Net:
    """The warm-start network of the library (see include/slar.h): FP32 parameters,
    forward, loss gradient and Adam training step run in the library's kernels."""

    def __init__(self, m: int, n0: int, n1: int, hidden: int = 32, max_batch: int = 16, stream=None):
        import torch
        self.lib = load()
        self.m, self.n0, self.n1, self.hidden = m, n0, n1, hidden
        self.NX = n0 * n1
        self.max_batch = max_batch
        self.np = net_param_count(m, hidden)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        st = self.lib.slar_net_create(m, hidden, n0, n1, max_batch, C.c_void_p(stream.cuda_stream), C.byref(h))
        if st != SLAR_OK:
            raise SlarError(st, "slar_net_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.slar_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != SLAR_OK:
            raise SlarError(st, what)

    def set_params(self, theta: np.ndarray):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        if t.size != self.np:
            raise ValueError(f"expected {self.np} parameters, got {t.size}")
        self._check(self.lib.slar_net_set_params(self.h, t.ctypes.data_as(C.c_void_p), self.np), "set_params")

    def get_params(self) -> np.ndarray:
        t = np.zeros(self.np, dtype=np.float32)
        self._check(self.lib.slar_net_get_params(self.h, t.ctypes.data_as(C.c_void_p), self.np), "get_params")
        return t

    def forward(self, x, y):
        """x: float32 CUDA [batch][2m][NX] -> y: float32 CUDA [batch][m+m^2][NX]."""
        b = x.shape[0]
        if not (1 <= b <= self.max_batch) or x.numel() != b * 2 * self.m * self.NX or \
                y.numel() != b * (self.m + self.m * self.m) * self.NX:
            raise ValueError("bad forward shapes")
        self._check(self.lib.slar_net_forward(self.h, C.c_void_p(_ptr(x)), x.shape[0], C.c_void_p(_ptr(y))),
                    "forward")

    def _check_batch(self, samples, n_probes, idx):
        """The library cannot see buffer sizes: check them here."""
        L = sample_floats(self.m, self.NX, n_probes)
        if samples.dim() != 2 or samples.shape[1] != L or samples.dtype.itemsize != 4:
            raise ValueError(f"samples must be float32 [n, {L}]")
        if idx.dtype.itemsize != 4 or idx.dim() != 1 or not (1 <= idx.shape[0] <= self.max_batch):
            raise ValueError("idx must be int32 [batch], 1 <= batch <= max_batch")
        if int(idx.min()) < 0 or int(idx.max()) >= samples.shape[0]:
            raise ValueError("sample index out of range")

    def loss_grad(self, samples, n_probes: int, idx, grad=None) -> float:
        self._check_batch(samples, n_probes, idx)
        if grad is not None and grad.numel() != self.np:
            raise ValueError("grad must hold every parameter")
        L = C.c_double()
        self._check(self.lib.slar_net_loss_grad(self.h, C.c_void_p(_ptr(samples)), n_probes,
                                                C.c_void_p(_ptr(idx)), idx.shape[0], C.byref(L),
                                                C.c_void_p(_ptr(grad))), "loss_grad")
        return L.value

    def train_step(self, samples, n_probes: int, idx, lr: float, want_loss: bool = False):
        self._check_batch(samples, n_probes, idx)
        L = C.c_double()
        self._check(self.lib.slar_net_train_step(self.h, C.c_void_p(_ptr(samples)), n_probes,
                                                 C.c_void_p(_ptr(idx)), idx.shape[0], C.c_float(lr),
                                                 C.byref(L) if want_loss else None), "train_step")
        return L.value if want_loss else None
