"""Adaptive cross approximation that rebuilds the HT tensor from sampled entries (the
HTACA step of SLAR, Sec. 3.1 "SLAR(F; a, dt, eps)" and Sec. 1).

Test infrastructure: part of the FP64 oracle, never called by the CUDA path.

The paper defers HTACA's details to earlier work; it states only that entries are sampled
"typically along fibers" without forming the full tensor and that the final step is the
HSVD truncation of Supp. B.1.  The reading implemented here (deterministic):

1. Cross approximation with partial pivoting of the matricisation A = F_(x | v) at the
   root split (rows = spatial multi-index, columns = velocity multi-index).  Every step
   samples one full row fibre and one full column fibre of A:
     r = A(i_k, :) - sum_{l<k} u_l[i_k] v_l,   j_k = argmax |r|,  v_k = r / r[j_k],
     u_k = A(:, j_k) - sum_{l<k} v_l[j_k] u_l,  i_{k+1} = argmax_{i not used} |u_k[i]|.
   Start row i_1 = 0 (f > 0 makes every row non-zero).  Stop when
   ||u_k|| ||v_k|| <= eps ||A_k||_F (running estimate) and the residual sampled on a fixed
   set of check rows confirms it, or k = cap, or when the residual row vanishes.
   Check rows: the q = min(8, M1) distinct rows floor(frac(c g) M1), c = 1, 2, ..., with
   g = (sqrt 5 - 1)/2 (golden-ratio sequence, spread over the spatial grid); their
   residuals R_c = A(c, :) - sum_l u_l[c] v_l are kept up to date, and the stop is
   accepted only if (M1 / q) sum_c ||R_c||^2 <= eps^2 ||A_k||_F^2; otherwise the next
   row pivot is the unused check row of largest residual.  (The rank-1 test alone only
   sees the pivot row: on weak Landau it stopped at rank 4 with a cross error of 84 eps.)
   Arg-max ties: values within a relative 1e-10 of the maximum are treated as equal and
   the lowest index wins, so that pivots are reproducible across implementations that
   round differently.
   Negligible rows: a residual row whose largest entry (over unused columns) is at most
   max(1e-14, eps / 100) of the first pivot's magnitude adds no term.  Below eps / 100 a
   pivot only resolves structure beneath the requested accuracy while multiplying rounding
   errors by 1 / |pivot| (the cross factor v = r / r[j]); at the 1e-14 floor the row is
   rounding noise -- data that repeat a row already crossed, as under the half-period
   shift symmetry of cos kx1 cos kx2, or data reproduced exactly -- and the pivot would
   depend on how an implementation rounds.  Such a row counts as a vanishing term for the
   stop test: the check rows decide between stopping and continuing from the unused check
   row of largest residual.
2. The factors A ~ U V^T are embedded exactly as an HT: d = 2: leaves U, V and root I;
   d = 4: identity leaves, B12[a,b,p] = U[(a,b),p], B34[c,e,q] = V[(c,e),q], root I.
2'. (Option, d = 4.)  Leaf bases of rank r_mu <= N_mu instead of the identity: each leaf
   unfolding of the cross factors -- one side weighted by the other side's triangular QR
   factor, so that its norm is ||A||_F -- is compressed by greedy column-pivoted QR to a
   residual of eps / (2 sqrt(2d - 3)) of ||A||_F (``compress_leaves``); the truncation then
   eigen-solves leaf Gram matrices of order r_mu instead of N_mu.
3. HSVD truncation (``ht.truncate``) with eps and the rank cap gives the new HT, whose
   leaf columns 0 are the leading mode singular vectors needed by the LoMaC weight.

The number of sampled entries per call is k (M1 + M2) + q M2 (check rows; none in replay).
"""
from __future__ import annotations

import math
from typing import Callable, Optional

import numpy as np

from . import ht as htmod

TIE_RTOL = 1e-10
NOISE_RTOL = 1e-14
N_CHECK = 8
GOLDEN = (math.sqrt(5.0) - 1.0) / 2.0


def check_rows(M1: int, q: int = N_CHECK):
    """The check rows of the stop test: distinct floor(frac(c g) M1), c = 1, 2, ..."""
    rows = []
    c = 1
    while len(rows) < min(q, M1) and c <= 64 * q + M1:
        i = int(math.floor(math.fmod(c * GOLDEN, 1.0) * M1))
        if i not in rows:
            rows.append(i)
        c += 1
    return rows


def argmax_tie(a: np.ndarray, excluded: Optional[np.ndarray] = None) -> int:
    """Index of max |a| (excluded positions ignored); near-ties go to the lowest index."""
    m = np.abs(a).astype(np.float64)
    if excluded is not None:
        m = m.copy()
        m[excluded] = -1.0
    top = m.max()
    if top < 0.0:
        return -1
    cand = np.nonzero(m >= top * (1.0 - TIE_RTOL))[0]
    return int(cand[0])


def aca(row_fn: Callable[[int], np.ndarray], col_fn: Callable[[int], np.ndarray], M1: int, M2: int,
        eps: float, kmax: int, pivots=None):
    """Partially pivoted cross approximation A ~ U V^T.

    row_fn(i) -> A(i, :) (length M2) and col_fn(j) -> A(:, j) (length M1) sample fibres.
    ``pivots`` (list of (i, j)) replays a given pivot sequence instead of choosing.
    Returns dict(U (M1,k), V (M2,k), I, J, entries, skipped) with `skipped` the number of
    negligible rows sampled without a term."""
    Us, Vs, I, J = [], [], [], []
    used_r = np.zeros(M1, dtype=bool)
    used_c = np.zeros(M2, dtype=bool)
    normA2 = 0.0
    i = 0 if pivots is None else pivots[0][0]
    n_entries = 0
    kmax = min(kmax, M1, M2)
    chk = check_rows(M1) if pivots is None else []
    R = np.stack([row_fn(c).astype(np.float64) for c in chk]) if chk else np.zeros((0, M2))
    n_entries += len(chk) * M2
    piv0 = None
    skipped = 0
    k = 0
    while k < kmax:
        if pivots is not None:
            if k >= len(pivots):
                break
            i = pivots[k][0]
        r = row_fn(i).astype(np.float64)
        n_entries += M2
        for l in range(len(Us)):
            r = r - Us[l][i] * Vs[l]
        used_r[i] = True
        if pivots is None:
            rmax = np.max(np.abs(np.where(used_c, 0.0, r)))
            if rmax == 0.0 and piv0 is None:
                break
            if piv0 is not None and rmax <= max(NOISE_RTOL, 0.01 * eps) * piv0:
                # a negligible row: no term; the check rows decide (as for a vanishing term)
                skipped += 1
                n2 = np.array([float(R[q] @ R[q]) for q in range(len(chk))])
                if not chk or M1 / len(chk) * float(np.sum(n2)) <= eps * eps * normA2:
                    break
                free = [q for q in range(len(chk)) if not used_r[chk[q]]]
                if not free:
                    break
                i = chk[max(free, key=lambda q: (n2[q], -q))]
                continue
            j = argmax_tie(r, used_c)
        else:
            j = pivots[k][1]
        piv = r[j]
        if piv == 0.0:
            break
        if piv0 is None:
            piv0 = abs(piv)
        v = r / piv
        c = col_fn(j).astype(np.float64)
        n_entries += M1
        for l in range(len(Us)):
            c = c - Vs[l][j] * Us[l]
        used_c[j] = True
        u = c
        # running Frobenius norm of the approximation (standard ACA estimate)
        cross = 0.0
        for l in range(len(Us)):
            cross += float(Us[l] @ u) * float(Vs[l] @ v)
        nu, nv = float(np.linalg.norm(u)), float(np.linalg.norm(v))
        normA2 = normA2 + 2.0 * cross + (nu * nv) ** 2
        Us.append(u)
        Vs.append(v)
        I.append(i)
        J.append(j)
        k += 1
        if pivots is None:
            for q, c in enumerate(chk):
                R[q] = R[q] - u[c] * v
            if nu * nv <= eps * np.sqrt(max(normA2, 0.0)):
                n2 = np.array([float(R[q] @ R[q]) for q in range(len(chk))])
                if M1 / len(chk) * float(np.sum(n2)) <= eps * eps * normA2:
                    break
                free = [q for q in range(len(chk)) if not used_r[chk[q]]]
                if not free:
                    break
                i = chk[max(free, key=lambda q: (n2[q], -q))]
                continue
            i = argmax_tie(u, used_r)
    k = len(Us)
    U = np.stack(Us, axis=1) if k else np.zeros((M1, 0))
    V = np.stack(Vs, axis=1) if k else np.zeros((M2, 0))
    return dict(U=U, V=V, I=I, J=J, entries=n_entries, skipped=skipped)


def top_rows(a: np.ndarray, excluded: np.ndarray, b: int):
    """The b rows of largest |a| outside `excluded`, in that order (each pick by argmax_tie:
    near-ties to the lowest index)."""
    ex = excluded.copy()
    out = []
    for _ in range(b):
        i = argmax_tie(a, ex)
        if i < 0:
            break
        out.append(i)
        ex[i] = True
    return out


def aca_block(rows_fn: Callable[[list], np.ndarray], cols_fn: Callable[[list], np.ndarray], M1: int, M2: int,
              eps: float, kmax: int, b: int):
    """Block cross approximation (the "next" row of the scope: rank-level parallel HTACA),
    A ~ U V^T with b row fibres and up to b column fibres sampled per step.

    rows_fn(list of i) -> A(i, :) stacked (len, M2); cols_fn(list of j) -> A(:, j) as (M1, len).
    Reading (the paper names HTACA's serial pivot steps as its bottleneck and defers the
    method): a step takes the rows I of its block -- row 0 and the first b - 1 other check
    rows at the start, then the b rows of largest |u| of the latest column residual outside
    the used rows (after a stop test that the check rows did not confirm, the unused check
    row of largest residual first) -- samples their residual rows R = A(I, :) - U(I) V^T at
    once, and pivots in them in order, exactly like partial pivoting restricted to I:
        row t of I: r = R[t] (already reduced by the block's earlier terms),
        negligible (as in ``aca``): no term;  else j_t = argmax |r|, v_t = r / r[j_t],
        and R[t'] -= R[t'][j_t] v_t for the later rows t' of the block.
    Then the accepted columns J are sampled at once, C = A(:, J) - U V(J)^T, and the column
    factors follow by forward substitution, u_t = C[:, t] - sum_{s<t} u_s v_s[j_t] (the
    residual column after the block's earlier terms).  The terms are accepted in order with
    the stop test of ``aca`` (rank-1 test confirmed on the check rows); the rest of a block
    after a confirmed stop is dropped.  With b = 1 this is ``aca``.
    Returns the same dict as ``aca``."""
    Us, Vs, I, J = [], [], [], []
    used_r = np.zeros(M1, dtype=bool)
    used_c = np.zeros(M2, dtype=bool)
    normA2 = 0.0
    kmax = min(kmax, M1, M2)
    chk = check_rows(M1)
    R = rows_fn(chk).astype(np.float64) if chk else np.zeros((0, M2))
    n_entries = len(chk) * M2
    piv0 = None
    skipped = 0
    next_rows = [0] + [c for c in chk if c != 0][: b - 1]

    def check_decision():
        """After a vanishing term or a passed rank-1 test: (stop, redirect row or None)."""
        n2 = np.array([float(R[q] @ R[q]) for q in range(len(chk))])
        if not chk or M1 / len(chk) * float(np.sum(n2)) <= eps * eps * normA2:
            return True, None
        free = [q for q in range(len(chk)) if not used_r[chk[q]]]
        if not free:
            return True, None
        return False, chk[max(free, key=lambda q: (n2[q], -q))]

    stop = False
    while not stop and len(Us) < kmax:
        rows = []
        for i in next_rows:
            if not used_r[i] and i not in rows:
                rows.append(i)
        rows = rows[: min(b, kmax - len(Us))]
        if not rows:
            break
        Rb = rows_fn(rows).astype(np.float64)
        n_entries += len(rows) * M2
        for l in range(len(Us)):
            Rb = Rb - np.outer(Us[l][rows], Vs[l])
        for i in rows:
            used_r[i] = True
        acc_rows, acc_cols, vs = [], [], []
        first_zero = False
        for t, i in enumerate(rows):
            r = Rb[t]
            rmax = float(np.max(np.abs(np.where(used_c, 0.0, r))))
            if rmax == 0.0 and piv0 is None:
                first_zero = True
                break
            if piv0 is not None and rmax <= max(NOISE_RTOL, 0.01 * eps) * piv0:
                skipped += 1
                continue
            j = argmax_tie(r, used_c)
            piv = r[j]
            if piv0 is None:
                piv0 = abs(piv)
            v = r / piv
            used_c[j] = True
            acc_rows.append(i)
            acc_cols.append(j)
            vs.append(v)
            for t2 in range(t + 1, len(rows)):
                Rb[t2] = Rb[t2] - Rb[t2][j] * v
        if first_zero:
            break
        redirect = None
        if not acc_cols:
            # every row of the block negligible: a vanishing term for the stop test
            stop, redirect = check_decision()
            if stop:
                break
            next_rows = [redirect] + top_rows(Us[-1], used_r | (np.arange(M1) == redirect), b - 1)
            continue
        C = cols_fn(acc_cols).astype(np.float64)
        n_entries += len(acc_cols) * M1
        for l in range(len(Us)):
            C = C - np.outer(Us[l], Vs[l][acc_cols])
        new_us = []
        for t in range(len(acc_cols)):
            u = C[:, t].copy()
            for s in range(t):
                u = u - new_us[s] * vs[s][acc_cols[t]]
            new_us.append(u)
        for t in range(len(acc_cols)):
            u, v = new_us[t], vs[t]
            cross = 0.0
            for l in range(len(Us)):
                cross += float(Us[l] @ u) * float(Vs[l] @ v)
            nu, nv = float(np.linalg.norm(u)), float(np.linalg.norm(v))
            normA2 = normA2 + 2.0 * cross + (nu * nv) ** 2
            Us.append(u)
            Vs.append(v)
            I.append(acc_rows[t])
            J.append(acc_cols[t])
            for q, cq in enumerate(chk):
                R[q] = R[q] - u[cq] * v
            if nu * nv <= eps * np.sqrt(max(normA2, 0.0)):
                stop, redirect = check_decision()
                if stop:
                    break
        if stop:
            break
        base = top_rows(Us[-1], used_r | (np.arange(M1) == redirect) if redirect is not None else used_r,
                        b - (1 if redirect is not None else 0))
        next_rows = ([redirect] if redirect is not None else []) + base
    k = len(Us)
    U = np.stack(Us, axis=1) if k else np.zeros((M1, 0))
    V = np.stack(Vs, axis=1) if k else np.zeros((M2, 0))
    return dict(U=U, V=V, I=I, J=J, entries=n_entries, skipped=skipped)


def embed(U: np.ndarray, V: np.ndarray, N) -> htmod.HT:
    """Exact HT of U V^T on the root split (step 2 of the module docstring)."""
    k = U.shape[1]
    if len(N) == 2:
        return htmod.HT(U=[U.copy(), V.copy()], Broot=np.eye(k))
    B12 = U.reshape(N[0], N[1], k)
    B34 = V.reshape(N[2], N[3], k)
    return htmod.HT(U=[np.eye(N[0]), np.eye(N[1]), np.eye(N[2]), np.eye(N[3])],
                    Broot=np.eye(k), B12=B12.copy(), B34=B34.copy())


def qrcp_basis(M: np.ndarray, tol: float):
    """Orthonormal basis of columns of M (n x m, in memory) chosen greedily by column
    pivoting (Businger-Golub): each step takes the column of largest residual norm (ties as
    in the cross approximation: within a relative 1e-10 of the maximum, the lowest index),
    normalises its residual against the basis so far (two Gram-Schmidt passes), and stops
    once the residual Frobenius norm ||M - Q Q^T M||_F is at most tol or the basis has
    min(n, m) columns.  Returns (Q (n x r), chosen column indices)."""
    n, m = M.shape
    Rm = np.array(M, dtype=np.float64, copy=True)
    Q = np.zeros((n, 0))
    cols = []
    used = np.zeros(m, dtype=bool)
    while Q.shape[1] < min(n, m):
        norms2 = np.einsum("ij,ij->j", Rm, Rm)
        if math.sqrt(float(norms2.sum())) <= tol:
            break
        j = argmax_tie(np.sqrt(norms2), used)
        q = Rm[:, j].copy()
        for _ in range(2):
            q = q - Q @ (Q.T @ q)
        nq = float(np.linalg.norm(q))
        if nq == 0.0:
            break
        q = q / nq
        Q = np.concatenate([Q, q[:, None]], axis=1)
        used[j] = True
        cols.append(int(j))
        Rm = Rm - np.outer(q, q @ Rm)
    return Q, cols


def compress_leaves(U: np.ndarray, V: np.ndarray, N, eps: float) -> htmod.HT:
    """HT with orthonormal leaf bases of rank r_mu <= N_mu for A = U V^T on the d = 4 root
    split (step 2' of the module docstring): the identity leaves of ``embed`` replaced by
    bases of the leaf unfoldings of the cross factors, chosen by ``qrcp_basis``.

    With V = Q_V R_V, W = U R_V^T (so A = W Q_V^T and ||W||_F = ||A||_F): the mode-x1 and
    mode-x2 unfoldings of W (as N0 x N1 x K) give Q0, Q1 at tolerance eps_l ||A||_F each, and
    C12 = W x_0 Q0^T x_1 Q1^T.  With C12 (as r0 r1 x K) = Q_C R_C and Z = Q_V R_C^T (so the
    compressed A' = (Q0 (x) Q1) Q_C Z^T and ||Z||_F = ||A'||_F): the mode-v1 and mode-v2
    unfoldings of Z give Q2, Q3, and C34 = Z x_0 Q2^T x_1 Q3^T.  The HT: leaves Q0..Q3,
    B12 = Q_C (r0, r1, K), B34 = C34 (r2, r3, K), root I_K.  Each projection removes at most
    eps_l of the norm it acts on, so ||A - HT|| <= ~4 eps_l ||A||_F; eps_l =
    eps / (2 sqrt(2d - 3)) keeps that below the eps of the truncation that follows."""
    if len(N) != 4:
        raise ValueError("leaf compression is for d = 4 (d = 2 leaves are the factors)")
    K = U.shape[1]
    n0, n1, n2, n3 = (int(x) for x in N)
    eps_l = eps / (2.0 * math.sqrt(5.0))
    if K == 0:
        return htmod.HT(U=[np.zeros((n, 0)) for n in (n0, n1, n2, n3)], Broot=np.zeros((0, 0)),
                        B12=np.zeros((0, 0, 0)), B34=np.zeros((0, 0, 0)))
    QV, RV = np.linalg.qr(V)
    W = (U @ RV.T).reshape(n0, n1, K)
    tol = eps_l * float(np.linalg.norm(W))
    Q0, _ = qrcp_basis(W.reshape(n0, n1 * K), tol)
    Q1, _ = qrcp_basis(np.transpose(W, (1, 0, 2)).reshape(n1, n0 * K), tol)
    C12 = np.einsum("abk,ax,by->xyk", W, Q0, Q1)
    r0, r1 = Q0.shape[1], Q1.shape[1]
    QC, RC = np.linalg.qr(C12.reshape(r0 * r1, K))
    kk = QC.shape[1]
    Z = (QV @ RC.T).reshape(n2, n3, kk)
    tol2 = eps_l * float(np.linalg.norm(Z))
    Q2, _ = qrcp_basis(Z.reshape(n2, n3 * kk), tol2)
    Q3, _ = qrcp_basis(np.transpose(Z, (1, 0, 2)).reshape(n3, n2 * kk), tol2)
    C34 = np.einsum("cek,cx,ey->xyk", Z, Q2, Q3)
    return htmod.HT(U=[Q0, Q1, Q2, Q3], Broot=np.eye(kk), B12=QC.reshape(r0, r1, kk), B34=C34)


def htaca(entry_fn: Callable[[np.ndarray], np.ndarray], N, eps: float, cap: int,
          pivots=None, return_info: bool = False, block: int = 1, leaf_compress: bool = False):
    """Build the HT of the tensor whose entries are entry_fn(idx (S, d)) from sampled row
    and column fibres of the root-split matricisation, then truncate (module docstring).
    block > 1: the block cross approximation (``aca_block``) with that many fibres per step;
    replayed pivots give the same cross approximation whatever the blocking.  leaf_compress
    (d = 4): orthonormal leaf bases of rank r_mu from the cross factors (``compress_leaves``)
    instead of identity leaves of order N_mu before the truncation."""
    d = len(N)
    half = d // 2
    Nl, Nr = N[:half], N[half:]
    M1, M2 = int(np.prod(Nl)), int(np.prod(Nr))
    left = np.stack(np.unravel_index(np.arange(M1), Nl), axis=1)
    right = np.stack(np.unravel_index(np.arange(M2), Nr), axis=1)

    def row_fn(i):
        idx = np.concatenate([np.repeat(left[i:i + 1], M2, axis=0), right], axis=1)
        return entry_fn(idx)

    def col_fn(j):
        idx = np.concatenate([left, np.repeat(right[j:j + 1], M1, axis=0)], axis=1)
        return entry_fn(idx)

    def rows_fn(rows):
        return np.stack([row_fn(i) for i in rows])

    def cols_fn(cols):
        return np.stack([col_fn(j) for j in cols], axis=1)

    if block > 1 and pivots is None:
        res = aca_block(rows_fn, cols_fn, M1, M2, eps, cap, block)
    else:
        res = aca(row_fn, col_fn, M1, M2, eps, cap, pivots)
    if leaf_compress and d == 4:
        full = compress_leaves(res["U"], res["V"], N, eps)
    else:
        full = embed(res["U"], res["V"], N)
    out, tinfo = htmod.truncate(full, eps, cap, return_info=True)
    if return_info:
        info = dict(aca_rank=res["U"].shape[1], pivots=list(zip(res["I"], res["J"])),
                    entries=res["entries"], ranks=tinfo["ranks"], skipped=res["skipped"])
        return out, info
    return out
