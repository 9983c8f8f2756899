"""Writes an oracle state in the library's checkpoint format (the layout slar_checkpoint
writes, include/slar.h), so that a GPU context can be restarted from any point of an oracle
trajectory with slar_restore.  Test helper: arrays come from the oracle only."""
import struct

import numpy as np

import convert

MAGIC = b"SLARCKPT"
VERSION = 2


def write_checkpoint(path, w, st):
    """w: the workload (grid, box); st: oracle stepper.State at the start of a step."""
    d = w.dx + w.dv
    lib = convert.to_lib(st.F)
    U = lib["U"]
    rank = [u.shape[1] for u in U] + [0] * (4 - d)
    if d == 4:
        rank[4:6] = [lib["B12"].shape[0], lib["B34"].shape[0]]
    else:
        rank += [0, 0]
    N = list(w.N) + [1] * (4 - d)
    lo = list(w.lo) + [0.0] * (4 - d)
    hi = list(w.hi) + [1.0] * (4 - d)
    has_corr = 1 if st.F.corr is not None else 0
    dts = list(st.dts) + [0.0, 0.0]
    hdr = struct.pack("=8si3i4i4d4d4i6i6idq2d", MAGIC, VERSION, d, w.dx, w.dv, *N, *lo, *hi,
                      0, st.step, 1, has_corr, *rank, *([0] * 6), st.n_i, 0, dts[0], dts[1])
    assert len(hdr) == 200
    nU = (w.dv + 2) * int(np.prod(w.N[:w.dx]))
    with open(path, "wb") as f:
        f.write(hdr)
        for u in U:
            f.write(np.ascontiguousarray(u, dtype=np.float64).tobytes())
        if d == 4:
            f.write(lib["B12"].astype(np.float64).tobytes())
            f.write(lib["B34"].astype(np.float64).tobytes())
        f.write(np.ascontiguousarray(lib["Broot"], dtype=np.float64).tobytes())
        if has_corr:
            terms = st.F.corr.terms
            dv = w.dv
            om = terms[0][1]
            qv = np.zeros((3, dv, w.N[w.dx]))
            for m in range(dv):
                qv[0, m] = om[m]
                qv[1, m] = terms[1 + m][1][m]
                qv[2, m] = terms[1 + dv + m][1][m]
            f.write(np.ascontiguousarray(st.F.corr.dC, dtype=np.float64).reshape(-1).tobytes())
            f.write(qv.tobytes())
        hist = list(st.hist) + [np.zeros_like(st.U)] * 2
        for arr in (st.U, hist[0], hist[1]):
            a = np.ascontiguousarray(arr, dtype=np.float64).reshape(-1)
            assert a.size == nU
            f.write(a.tobytes())
