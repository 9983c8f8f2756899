"""Block-circulant preconditioning of the macroscopic Newton-Krylov solve, and the
preconditioned JFNK used by the learned warm start.

Test infrastructure: part of the FP64 oracle, never called by the CUDA path.

The paper solves G(U) = 0 of Sec. 3.2.3 by JFNK without a preconditioner.  This module
adds one, as part of the warm-start addition:

* The Jacobian J of G at the initial guess is probed with one impulse per conserved
  component: r_c = J (e_c delta_0), a finite-difference Jacobian-vector product with the
  step of Knoll and Keyes (2004).  For a spatially invariant operator J is block-circulant
  and r_c is its c-th block column, so with R(k)[c', c] = DFT(r_c[c'])(k) the operator acts
  on Fourier modes as the (dv+2) x (dv+2) block R(k).  The preconditioner applies R(k)^{-1}
  mode by mode (the block-circulant approximation of T. Chan's circulant preconditioners).
  A block whose Gauss-Jordan pivot falls below 1e-14 times its largest entry is replaced
  by the identity.
* Right preconditioning: GMRES solves (J P) y = -G, the Newton correction is P y; the
  Newton stop test and the line of the plain method are unchanged, so the converged U is
  judged by the same residual.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np

from . import macro

EPS_MACH = 2.0 ** -52
PIVOT_FLOOR = 1e-14


def fd_jv(Gfun, U: np.ndarray, G0: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Finite-difference J v = (G(U + h v) - G(U)) / h, h = sqrt(eps)(1+||U||)/||v||."""
    vn = float(np.linalg.norm(v))
    if vn == 0.0:
        return np.zeros_like(v)
    h = math.sqrt(EPS_MACH) * (1.0 + float(np.linalg.norm(U))) / vn
    return (Gfun(U + h * v) - G0) / h


def gauss_jordan_inverse(A: np.ndarray) -> np.ndarray:
    """Inverse of a small complex matrix by Gauss-Jordan elimination with partial pivoting;
    the identity if a pivot is below PIVOT_FLOOR * max|A|."""
    m = A.shape[0]
    M = np.concatenate([A.astype(complex), np.eye(m, dtype=complex)], axis=1)
    scale = float(np.max(np.abs(A)))
    for col in range(m):
        piv = col + int(np.argmax(np.abs(M[col:, col])))
        if not (abs(M[piv, col]) > PIVOT_FLOOR * scale):
            return np.eye(m, dtype=complex)
        if piv != col:
            M[[col, piv]] = M[[piv, col]]
        M[col] = M[col] / M[col, col]
        for r in range(m):
            if r != col:
                M[r] = M[r] - M[r, col] * M[col]
    return M[:, m:]


def circulant_blocks(Gfun, U: np.ndarray, G0: np.ndarray, shape2d) -> np.ndarray:
    """Inverse symbol P(k) (n0, n1, m, m) of the block-circulant approximation of J at U."""
    m = U.shape[0]
    R = np.zeros(tuple(shape2d) + (m, m), dtype=complex)
    for c in range(m):
        e = np.zeros_like(U)
        e[c, 0] = 1.0
        r = fd_jv(Gfun, U, G0, e)
        for c2 in range(m):
            R[..., c2, c] = np.fft.fft2(r[c2].reshape(shape2d))
    P = np.empty_like(R)
    for idx in np.ndindex(*shape2d):
        P[idx] = gauss_jordan_inverse(R[idx])
    return P


def apply_circulant(P: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Apply the mode-wise blocks P(k) to y (m, NX)."""
    m = y.shape[0]
    shape2d = P.shape[:2]
    Yh = np.stack([np.fft.fft2(y[c].reshape(shape2d)) for c in range(m)], axis=-1)
    Zh = np.einsum("...ij,...j->...i", P, Yh)
    return np.stack([np.real(np.fft.ifft2(Zh[..., c])).reshape(-1) for c in range(m)])


@dataclass
class PJFNKStats:
    newton: int = 0
    krylov: int = 0
    residual: float = 0.0
    converged: bool = False


def jfnk_right(Gfun: Callable[[np.ndarray], np.ndarray], U0: np.ndarray, tol_abs: float,
               krylov_tol: float, Papply: Optional[Callable[[np.ndarray], np.ndarray]],
               restart: int = 30, newton_max: int = 20, krylov_max: int = 200):
    """JFNK with right preconditioning P (None = identity, which is macro.jfnk)."""
    st = PJFNKStats()
    U = U0.copy()
    shape = U.shape
    P = (lambda y: y) if Papply is None else (lambda y: Papply(y.reshape(shape)).reshape(-1))
    Gu = Gfun(U)
    for _ in range(newton_max):
        st.residual = float(np.max(np.abs(Gu)))
        if st.residual <= tol_abs:
            st.converged = True
            break
        G0 = Gu

        def A(y):
            return fd_jv(Gfun, U, G0, P(y).reshape(shape)).reshape(-1)

        y, its = macro.gmres(A, -Gu.reshape(-1), krylov_tol, restart, krylov_max)
        st.krylov += its
        st.newton += 1
        U = U + P(y).reshape(shape)
        Gu = Gfun(U)
    else:
        st.residual = float(np.max(np.abs(Gu)))
        st.converged = st.residual <= tol_abs
    return U, st
