"""Hierarchical-Tucker (HT) tensors for the two dimension trees of the method (Sec. 3.1).

Test infrastructure: part of the FP64 oracle, never called by the CUDA path.

Trees (leaves numbered in the dimension order x1..x_dx, v1..v_dv):

* d = 2 (1D-1V):  root{0, 1}.  Entry F(i0, i1) = U0[i0] . Broot . U1[i1]^T.
* d = 4 (2D-2V):  root{12{0,1}, 34{2,3}}.
      c12[p] = sum_ab B12[a,b,p] U0[i0,a] U1[i1,b],  c34[q] likewise with B34, U2, U3,
      F(i0..i3) = c12 . Broot . c34.

Leaf bases U_mu are (N_mu, r_mu); transfer tensors B12 (r0, r1, r12), B34 (r2, r3, r34);
the root matrix Broot is (r0, r1) for d = 2 and (r12, r34) for d = 4.

A state of the LoMaC-corrected method also carries a separable correction
sum_k dC_k(x) (x) Q_k(v) (Eq. LoMaC_update_discrete), kept exactly (see ``Correction``).
"""
from __future__ import annotations

import copy
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Correction:
    """Separable LoMaC correction sum_k dC_k(x) (x) Q_k(v) added to an HT tensor.

    ``dC`` is (dv+2, prod N_x) (row-major spatial index, x1 slowest).  ``terms`` lists the
    separable velocity pieces as (k, [vec_mu for mu in 0..dv-1]) -- Q_2 is a sum of dv
    separable pieces, Q_0 and Q_{1,mu} are single pieces (Supp. B.2)."""
    dC: np.ndarray
    terms: list


@dataclass
class HT:
    U: List[np.ndarray]
    Broot: np.ndarray
    B12: Optional[np.ndarray] = None
    B34: Optional[np.ndarray] = None
    corr: Optional[Correction] = None

    @property
    def d(self) -> int:
        return len(self.U)

    @property
    def N(self):
        return tuple(u.shape[0] for u in self.U)

    def ranks(self):
        r = [u.shape[1] for u in self.U]
        if self.d == 4:
            r += [self.B12.shape[2], self.B34.shape[2]]
        return r

    def copy(self) -> "HT":
        return copy.deepcopy(self)

    def without_correction(self) -> "HT":
        h = copy.copy(self)
        h.corr = None
        return h


def from_raw(raw) -> HT:
    """Wrap raw factors (e.g. ``inputs.RandomHT``) as an HT."""
    return HT(U=[np.array(u, dtype=np.float64) for u in raw.U],
              Broot=np.array(raw.Broot, dtype=np.float64),
              B12=None if raw.B12 is None else np.array(raw.B12, dtype=np.float64),
              B34=None if raw.B34 is None else np.array(raw.B34, dtype=np.float64))


def from_terms(factors) -> HT:
    """Exact HT of a sum of separable terms f = sum_t prod_mu factors[t][mu] (used for the
    analytic initial data of Sec. 4).  Leaves stack the term factors as columns; the
    transfer tensors are 'diagonal' (B[a,b,p] = 1 iff a = b = p); the root is the identity."""
    T = len(factors)
    d = len(factors[0])
    U = [np.stack([factors[t][m] for t in range(T)], axis=1).astype(np.float64) for m in range(d)]
    I = np.eye(T)
    if d == 2:
        return HT(U=U, Broot=I)
    D = np.zeros((T, T, T))
    for t in range(T):
        D[t, t, t] = 1.0
    return HT(U=U, Broot=I, B12=D.copy(), B34=D.copy())


# ----------------------------------------------------------------------------------------
# entries and densification
# ----------------------------------------------------------------------------------------

def contract_tree(ht: HT, c: List[np.ndarray]) -> np.ndarray:
    """Contract per-entry leaf row vectors c[mu] (S, r_mu) up the dimension tree to the
    root scalar (Sec. 3.1: leaf vectors contracted with the transfer tensors recursively;
    O(d r^3) per entry).  Returns (S,)."""
    if ht.d == 2:
        return np.einsum("sa,ab,sb->s", c[0], ht.Broot, c[1])
    c12 = np.einsum("sa,sb,abp->sp", c[0], c[1], ht.B12)
    c34 = np.einsum("sc,se,ceq->sq", c[2], c[3], ht.B34)
    return np.einsum("sp,pq,sq->s", c12, ht.Broot, c34)


def spatial_linear_index(idx_x: np.ndarray, Nx) -> np.ndarray:
    """Row-major linear index of spatial multi-indices (x1 slowest)."""
    lin = np.zeros(idx_x.shape[0], dtype=np.int64)
    for m in range(len(Nx)):
        lin = lin * Nx[m] + idx_x[:, m]
    return lin


def correction_entries(corr: Correction, idx: np.ndarray, dx: int, N) -> np.ndarray:
    """Entries of the separable correction at grid index tuples."""
    lin = spatial_linear_index(idx[:, :dx], N[:dx])
    out = np.zeros(idx.shape[0])
    for k, vecs in corr.terms:
        t = corr.dC[k][lin].copy()
        for m, vec in enumerate(vecs):
            t = t * vec[idx[:, dx + m]]
        out = out + t
    return out


def entries(ht: HT, idx: np.ndarray) -> np.ndarray:
    """HT entries at integer grid tuples idx (S, d): leaf rows, then the tree contraction,
    plus the separable correction if the state carries one."""
    idx = np.asarray(idx, dtype=np.int64)
    c = [ht.U[m][idx[:, m]] for m in range(ht.d)]
    out = contract_tree(ht, c)
    if ht.corr is not None:
        out = out + correction_entries(ht.corr, idx, ht.d // 2, ht.N)
    return out


def densify(ht: HT) -> np.ndarray:
    """Full tensor of an HT (tiny grids only)."""
    if ht.d == 2:
        F = ht.U[0] @ ht.Broot @ ht.U[1].T
    else:
        P12 = np.einsum("ia,jb,abp->ijp", ht.U[0], ht.U[1], ht.B12)
        P34 = np.einsum("kc,le,ceq->klq", ht.U[2], ht.U[3], ht.B34)
        F = np.einsum("ijp,pq,klq->ijkl", P12, ht.Broot, P34)
    if ht.corr is not None:
        N = ht.N
        dx = ht.d // 2
        grids = np.meshgrid(*[np.arange(n) for n in N], indexing="ij")
        idx = np.stack([g.reshape(-1) for g in grids], axis=1)
        F = F + correction_entries(ht.corr, idx, dx, N).reshape(N)
    return F


def frob_norm(ht: HT) -> float:
    """Frobenius norm of the HT part (orthogonalise, then the root's norm)."""
    return float(np.linalg.norm(orthogonalize(ht).Broot))


# ----------------------------------------------------------------------------------------
# orthogonalisation and HSVD truncation (Supp. B.1: the final HTACA step)
# ----------------------------------------------------------------------------------------

def _qr(A: np.ndarray):
    Q, R = np.linalg.qr(A, mode="reduced")
    return Q, R


def orthogonalize(ht: HT) -> HT:
    """Orthonormal leaf bases and orthonormal internal frames; the root absorbs the rest.
    Leaves: U = Q R, R pushed into the parent.  Internal node t (d = 4): reshape B_t to
    (r_{t1} r_{t2}, r_t), QR, push R_t into the root."""
    Qs, Rs = zip(*[_qr(u) for u in ht.U])
    Qs, Rs = list(Qs), list(Rs)
    if ht.d == 2:
        return HT(U=Qs, Broot=Rs[0] @ ht.Broot @ Rs[1].T)
    B12 = np.einsum("xa,yb,abp->xyp", Rs[0], Rs[1], ht.B12)
    B34 = np.einsum("xc,ye,ceq->xyq", Rs[2], Rs[3], ht.B34)
    r0, r1, r12 = B12.shape
    r2, r3, r34 = B34.shape
    Q12, R12 = _qr(B12.reshape(r0 * r1, r12))
    Q34, R34 = _qr(B34.reshape(r2 * r3, r34))
    Broot = R12 @ ht.Broot @ R34.T
    return HT(U=Qs, Broot=Broot, B12=Q12.reshape(r0, r1, -1), B34=Q34.reshape(r2, r3, -1))


def node_gramians(h: HT):
    """Gram matrices of the node matricisations of an orthogonalised HT, expressed in the
    node bases, computed from the root down.  Returns a dict node -> symmetric matrix."""
    if h.d == 2:
        return {0: h.Broot @ h.Broot.T, 1: h.Broot.T @ h.Broot}
    G12 = h.Broot @ h.Broot.T
    G34 = h.Broot.T @ h.Broot
    G0 = np.einsum("abp,pq,xbq->ax", h.B12, G12, h.B12)
    G1 = np.einsum("abp,pq,ayq->by", h.B12, G12, h.B12)
    G2 = np.einsum("cep,pq,xeq->cx", h.B34, G34, h.B34)
    G3 = np.einsum("cep,pq,cyq->ey", h.B34, G34, h.B34)
    return {0: G0, 1: G1, 2: G2, 3: G3, 12: G12, 34: G34}


def _sorted_eig(G: np.ndarray):
    lam, S = np.linalg.eigh(0.5 * (G + G.T))
    order = np.argsort(lam)[::-1]
    return np.maximum(lam[order], 0.0), S[:, order]


def choose_rank(lam: np.ndarray, thresh2: float, cap: int) -> int:
    """Smallest k with sum_{i >= k} lam_i <= thresh2, then capped at ``cap`` (and >= 1)."""
    tail = np.concatenate([np.cumsum(lam[::-1])[::-1], [0.0]])
    k = int(np.argmax(tail <= thresh2))
    return max(1, min(k, cap, lam.shape[0]))


def truncate(ht: HT, eps: float, cap: int, return_info: bool = False):
    """HSVD truncation of an HT tensor (the final step of HTACA, Supp. B.1).

    Orthogonalise; form the node Gram matrices from the root down; eigendecompose them
    with eigenvalues in descending order; keep at every node the smallest rank whose
    discarded eigenvalue sum is at most (eps ||F||)^2 / (2d - 3) (so that the total error
    is at most eps ||F|| by the HSVD bound), capped at ``cap``; project leaves to root.
    The two children of the root share one matricisation and keep one common rank.
    Afterwards column 0 of every leaf basis is the leading left singular vector of the
    corresponding mode matricisation of the input (Supp. B.1).  The correction part of a
    state is not touched (it is never truncated).
    """
    h = orthogonalize(ht)
    G = node_gramians(h)
    normF2 = float(np.sum(h.Broot ** 2))
    thresh2 = (eps ** 2) * normF2 / (2 * h.d - 3)
    eig = {t: _sorted_eig(g) for t, g in G.items()}
    info = {}
    if h.d == 2:
        k = min(choose_rank(eig[0][0], thresh2, cap), eig[1][0].shape[0])
        S0 = eig[0][1][:, :k]
        S1 = eig[1][1][:, :k]
        out = HT(U=[h.U[0] @ S0, h.U[1] @ S1], Broot=S0.T @ h.Broot @ S1)
        info["ranks"] = [k, k]
    else:
        ks = {m: choose_rank(eig[m][0], thresh2, cap) for m in range(4)}
        k12 = min(choose_rank(eig[12][0], thresh2, cap), eig[34][0].shape[0])
        S = {m: eig[m][1][:, :ks[m]] for m in range(4)}
        S12 = eig[12][1][:, :k12]
        S34 = eig[34][1][:, :k12]
        U = [h.U[m] @ S[m] for m in range(4)]
        B12 = np.einsum("abp,ax,by,pz->xyz", h.B12, S[0], S[1], S12)
        B34 = np.einsum("ceq,cx,ey,qz->xyz", h.B34, S[2], S[3], S34)
        out = HT(U=U, Broot=S12.T @ h.Broot @ S34, B12=B12, B34=B34)
        info["ranks"] = [ks[0], ks[1], ks[2], ks[3], k12, k12]
    out.corr = ht.corr
    info["norm"] = np.sqrt(normF2)
    if return_info:
        return out, info
    return out
