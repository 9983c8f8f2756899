"""Layout conversions between the oracle's HT (B[a, b, p]) and the library's host view
([p][a][b] transfer tensors; correction as (dC, omega/q1/q2 vectors)).  Test helper."""
import numpy as np

from oracle import ht as htmod


def to_lib(h: htmod.HT) -> dict:
    out = dict(U=[np.ascontiguousarray(u) for u in h.U], Broot=np.ascontiguousarray(h.Broot))
    if h.d == 4:
        out["B12"] = np.ascontiguousarray(np.transpose(h.B12, (2, 0, 1)))
        out["B34"] = np.ascontiguousarray(np.transpose(h.B34, (2, 0, 1)))
    return out


def from_lib(ex: dict) -> htmod.HT:
    h = htmod.HT(U=[u.copy() for u in ex["U"]], Broot=ex["Broot"].copy())
    if ex["d"] == 4:
        h.B12 = np.ascontiguousarray(np.transpose(ex["B12"], (1, 2, 0)))
        h.B34 = np.ascontiguousarray(np.transpose(ex["B34"], (1, 2, 0)))
    if ex.get("has_corr"):
        h.corr = correction_from_qv(ex["dC"], ex["qv"])
    return h


def correction_from_qv(dC, qv) -> htmod.Correction:
    """Oracle correction whose separable pieces are Q0 = (x)omega, Q1_mu, Q2 (Supp. B.2)
    built from library vectors qv[f][mu] (f: omega, q1, q2)."""
    dv = qv.shape[1]
    om = [qv[0, m] for m in range(dv)]
    terms = [(0, list(om))]
    for m in range(dv):
        terms.append((1 + m, [qv[1, o] if o == m else om[o] for o in range(dv)]))
    for m in range(dv):
        terms.append((1 + dv, [qv[2, o] if o == m else om[o] for o in range(dv)]))
    return htmod.Correction(dC=np.array(dC), terms=terms)
