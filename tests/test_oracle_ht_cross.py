"""Oracle pins: HT orthogonalisation, HSVD truncation and the cross approximation
(Supp. B.1; the HTACA reading)."""
import math

import numpy as np
import pytest

from oracle import cross, sl
from oracle import ht as htmod
from paper_2606_29027_b300 import inputs


def _dense(h):
    return htmod.densify(h)


@pytest.mark.parametrize("N,ranks", [((9, 11), (6, 5)), ((6, 7, 5, 8), (5, 6, 4, 5, 7, 6))])
def test_orthogonalize_preserves_tensor(N, ranks):
    h = htmod.from_raw(inputs.random_ht(N, ranks, 3, smooth=False))
    o = htmod.orthogonalize(h)
    assert np.allclose(_dense(o), _dense(h), atol=1e-12 * np.abs(_dense(h)).max())
    for u in o.U:
        assert np.allclose(u.T @ u, np.eye(u.shape[1]), atol=1e-13)
    if len(N) == 4:
        for B in (o.B12, o.B34):
            M = B.reshape(-1, B.shape[2])
            assert np.allclose(M.T @ M, np.eye(M.shape[1]), atol=1e-13)


def test_truncation_matches_eckart_young_in_2d():
    """For d = 2 the HSVD is the matrix SVD: the truncation error equals the tail of the
    singular values (Eckart-Young), computed here by numpy's SVD of the dense matrix."""
    h = htmod.from_raw(inputs.random_ht((20, 24), (9, 9), 4, smooth=False))
    F = _dense(h)
    s = np.linalg.svd(F, compute_uv=False)
    for cap in (2, 5, 8):
        t = htmod.truncate(h, 1e-16, cap)
        err = np.linalg.norm(F - _dense(t))
        assert err == pytest.approx(np.sqrt(np.sum(s[cap:] ** 2)), rel=1e-9)


@pytest.mark.parametrize("eps", [1e-1, 3e-2, 1e-3])
def test_truncation_error_bound_4d(eps):
    """||F - F~|| <= eps ||F|| (HSVD bound with the per-node threshold eps^2 ||F||^2/(2d-3))."""
    N = (7, 8, 9, 6)
    h = htmod.from_raw(inputs.random_ht(N, (6, 6, 6, 6, 8, 8), 11, smooth=True))
    F = _dense(h)
    t, info = htmod.truncate(h, eps, 64, return_info=True)
    err = np.linalg.norm(F - _dense(t))
    assert err <= eps * np.linalg.norm(F) * (1 + 1e-12)
    assert max(info["ranks"]) <= 8


def test_truncation_leading_singular_vector():
    """After HSVD truncation column 0 of every leaf equals (up to sign) the leading left
    singular vector of the dense mode matricisation (Supp. B.1)."""
    N = (6, 7, 8, 9)
    h = htmod.from_raw(inputs.random_ht(N, (5, 5, 5, 5, 6, 6), 21, smooth=False))
    F = _dense(h)
    t = htmod.truncate(h, 1e-3, 64)
    for mu in range(4):
        A = np.moveaxis(F, mu, 0).reshape(N[mu], -1)
        u1 = np.linalg.svd(A, full_matrices=False)[0][:, 0]
        assert abs(float(t.U[mu][:, 0] @ u1)) == pytest.approx(1.0, abs=1e-10)
        assert np.allclose(t.U[mu].T @ t.U[mu], np.eye(t.U[mu].shape[1]), atol=1e-13)


def test_truncation_cap():
    h = htmod.from_raw(inputs.random_ht((6, 7, 8, 9), (5, 5, 5, 5, 6, 6), 2, smooth=False))
    t, info = htmod.truncate(h, 1e-14, 3, return_info=True)
    assert max(info["ranks"]) == 3


@pytest.mark.parametrize("N,ranks", [((24, 30), (3, 4)), ((6, 7, 5, 8), (2, 3, 3, 2, 3, 3))])
def test_cross_exact_recovery_of_low_rank(N, ranks):
    """HTACA reproduces an exactly low-rank tensor from sampled fibres (eps -> 1e-13)."""
    h = htmod.from_raw(inputs.random_ht(N, ranks, 8, smooth=False))
    F = _dense(h)
    out, info = cross.htaca(lambda idx: htmod.entries(h, idx), N, 1e-13, 64, return_info=True)
    assert np.linalg.norm(_dense(out) - F) <= 1e-10 * np.linalg.norm(F)
    M1 = int(np.prod(N[: len(N) // 2]))
    M2 = int(np.prod(N[len(N) // 2:]))
    # k terms, the check rows, and the rounding-level row that ends an exact reproduction
    assert info["entries"] == (info["aca_rank"] * (M1 + M2) + len(cross.check_rows(M1)) * M2
                               + info["skipped"] * M2)
    assert info["skipped"] <= 1
    # root-split rank of the data is the ACA rank bound
    rr = np.linalg.matrix_rank(F.reshape(M1, M2), tol=1e-9 * np.abs(F).max())
    assert info["aca_rank"] <= rr + 1


def test_cross_on_matrix_matches_svd_accuracy():
    """On a smooth kernel matrix the cross approximation reaches the requested relative
    accuracy within a small factor of the optimal (SVD) error of the same rank."""
    x = np.linspace(0, 1, 60)
    y = np.linspace(0, 2, 70)
    A = 1.0 / (1.0 + (x[:, None] - y[None, :]) ** 2) + 0.1 * np.cos(3 * x)[:, None]
    for eps in (1e-3, 1e-6, 1e-9):
        res = cross.aca(lambda i: A[i], lambda j: A[:, j], 60, 70, eps, 60)
        err = np.linalg.norm(A - res["U"] @ res["V"].T) / np.linalg.norm(A)
        assert err <= 10 * eps
        k = res["U"].shape[1]
        s = np.linalg.svd(A, compute_uv=False)
        assert k <= np.count_nonzero(s > 1e-3 * eps * s[0]) + 2


def test_cross_pivot_replay_reproduces():
    N = (12, 14)
    h = htmod.from_raw(inputs.random_ht(N, (5, 5), 9, smooth=True))
    fn = lambda idx: htmod.entries(h, idx)
    a, ia = cross.htaca(fn, N, 1e-8, 16, return_info=True)
    b, ib = cross.htaca(fn, N, 1e-8, 16, pivots=ia["pivots"], return_info=True)
    assert ia["pivots"] == ib["pivots"]
    assert np.allclose(_dense(a), _dense(b), atol=1e-14)


def test_argmax_tie_rule():
    a = np.array([1.0, -3.0, 3.0 * (1 - 1e-13), 2.0, -3.0])
    assert cross.argmax_tie(a) == 1
    ex = np.zeros(5, dtype=bool)
    ex[1] = True
    assert cross.argmax_tie(a, ex) == 2


def test_htaca_of_sl_update_close_to_truncated_dense():
    """SLAR(F): cross approximation of the SL-updated tensor is within a small multiple of
    eps of the dense SL step (brute force) on a tiny 2D-2V grid."""
    N = (10, 10, 12, 12)
    g = sl.PhaseGrid(2, 2, N, (0, 0, -5, -5), (4 * math.pi, 4 * math.pi, 5, 5))
    w = inputs.landau_2d2v(n=10, alpha=0.3)
    w.N, w.lo, w.hi = N, g.lo, g.hi
    F0 = htmod.truncate(htmod.from_terms(inputs.initial_factors(w)), 1e-12, 20)
    E = inputs.random_field(N[:2], 2, 0.3, seed=2)
    eps = 1e-6
    out = cross.htaca(lambda idx: sl.sl_eval(F0, E, 0.4, idx, g), N, eps, 40)
    dense = sl.dense_sl_step(htmod.densify(F0), E, 0.4, g)
    assert np.linalg.norm(_dense(out) - dense) <= 10 * eps * np.linalg.norm(dense)


def test_cross_stop_rule_catches_missed_structure():
    """First SLAR call of 2D2V weak Landau at 32^4 (eps 1e-5): the cross approximation of
    the SL-updated tensor is within eps of the dense SL update.  The rank-1 stop test alone
    stopped this call at rank 4 with an error of about 84 eps."""
    from oracle import sl, stepper
    w = inputs.landau_2d2v(n=32, cap=32)
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=1e-5, cap=w.rank_cap, lomac=False)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)
    E = stepper.field_of(st.F, g, st.n_i)
    ref = sl.dense_sl_step(htmod.densify(st.F), E, w.dt / 3, g)
    G, info = stepper.slar(st.F, E, w.dt / 3, g, prm)
    err = np.linalg.norm(htmod.densify(G) - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, (info["aca_rank"], err)


def test_check_rows_are_distinct_and_spread():
    for M1 in (1, 5, 64, 4096):
        rows = cross.check_rows(M1)
        assert len(rows) == min(8, M1) == len(set(rows))
        assert all(0 <= r < M1 for r in rows)
    r = sorted(cross.check_rows(4096))
    assert max(np.diff([0] + r + [4096])) < 4096 / 3


def test_rounding_level_row_is_skipped():
    """Two identical rows (rows 0 and 7, both of the largest magnitude): after the first
    term, row 7's residual is rounding noise, and the column residual points at it.  The
    cross approximation takes no pivot there (the pivot would be noise) and recovers the
    rank-2 matrix with exactly two terms from other rows; the pivots replay to the same
    result."""
    rng = np.random.default_rng(4)
    M1, M2 = 20, 30
    a = rng.uniform(-1, 1, M1)
    c = rng.uniform(-1, 1, M1)
    a[0] = a[7] = 3.0
    c[7] = c[0]
    b = rng.uniform(0.5, 1.0, M2)
    d = rng.uniform(-1, 1, M2)
    A = np.outer(a, b) + 0.3 * np.outer(c, d)
    assert np.array_equal(A[0], A[7])
    res = cross.aca(lambda i: A[i].copy(), lambda j: A[:, j].copy(), M1, M2, 1e-13, 10)
    assert res["U"].shape[1] == 2
    assert 7 not in res["I"][1:] and res["skipped"] >= 1
    assert np.linalg.norm(res["U"] @ res["V"].T - A) <= 1e-13 * np.linalg.norm(A)
    rep = cross.aca(lambda i: A[i].copy(), lambda j: A[:, j].copy(), M1, M2, 1e-13, 10,
                    pivots=list(zip(res["I"], res["J"])))
    assert np.allclose(rep["U"] @ rep["V"].T, res["U"] @ res["V"].T, rtol=0, atol=1e-15 * np.abs(A).max())


# ---------------------------------------------------------------- block cross approximation

def _matrix_fns(A):
    return (lambda rows: A[rows].copy(), lambda cols: A[:, cols].copy(),
            lambda i: A[i].copy(), lambda j: A[:, j].copy())


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_block_of_one_is_the_classical_cross(eps):
    """b = 1: the same pivots, entries and factors as the classical partial pivoting."""
    x = np.linspace(0, 1, 60)
    y = np.linspace(0, 2, 70)
    A = 1.0 / (1.0 + (x[:, None] - y[None, :]) ** 2) + 0.1 * np.cos(3 * x)[:, None]
    rf, cf, r1, c1 = _matrix_fns(A)
    a = cross.aca(r1, c1, 60, 70, eps, 60)
    b = cross.aca_block(rf, cf, 60, 70, eps, 60, 1)
    assert a["I"] == b["I"] and a["J"] == b["J"] and a["entries"] == b["entries"]
    assert np.allclose(a["U"] @ a["V"].T, b["U"] @ b["V"].T, rtol=0, atol=1e-15 * np.abs(A).max())


@pytest.mark.parametrize("b", [2, 4, 8])
@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_block_cross_accuracy_near_svd(b, eps):
    """Blocks of b fibres reach the requested accuracy (within 10 eps, as the classical
    cross approximation) with a rank within two of the SVD's numerical rank at 1e-3 eps."""
    x = np.linspace(0, 1, 60)
    y = np.linspace(0, 2, 70)
    A = 1.0 / (1.0 + (x[:, None] - y[None, :]) ** 2) + 0.1 * np.cos(3 * x)[:, None]
    rf, cf, _, _ = _matrix_fns(A)
    res = cross.aca_block(rf, cf, 60, 70, eps, 60, b)
    err = np.linalg.norm(A - res["U"] @ res["V"].T) / np.linalg.norm(A)
    assert err <= 10 * eps
    s = np.linalg.svd(A, compute_uv=False)
    assert res["U"].shape[1] <= np.count_nonzero(s > 1e-3 * eps * s[0]) + 2 + (b - 1)
    # every step's pivot pairs are distinct rows and columns
    assert len(set(res["I"])) == len(res["I"]) and len(set(res["J"])) == len(res["J"])


@pytest.mark.parametrize("b", [2, 4])
@pytest.mark.parametrize("N,ranks", [((24, 30), (3, 4)), ((6, 7, 5, 8), (2, 3, 3, 2, 3, 3))])
def test_block_cross_exact_recovery(b, N, ranks):
    h = htmod.from_raw(inputs.random_ht(N, ranks, 8, smooth=False))
    F = _dense(h)
    out, info = cross.htaca(lambda idx: htmod.entries(h, idx), N, 1e-13, 64, return_info=True, block=b)
    assert np.linalg.norm(_dense(out) - F) <= 1e-10 * np.linalg.norm(F)
    M1 = int(np.prod(N[: len(N) // 2]))
    M2 = int(np.prod(N[len(N) // 2:]))
    rr = np.linalg.matrix_rank(F.reshape(M1, M2), tol=1e-9 * np.abs(F).max())
    assert info["aca_rank"] <= rr + b


@pytest.mark.parametrize("b", [2, 4])
def test_block_pivots_replay_through_the_classical_path(b):
    """The cross approximation is fixed by its pivot pairs whatever the blocking: replaying
    a block run's pivots one at a time gives the same approximation to rounding (what the
    GPU's replay mode relies on)."""
    N = (12, 14)
    h = htmod.from_raw(inputs.random_ht(N, (5, 5), 9, smooth=True))
    fn = lambda idx: htmod.entries(h, idx)
    x = np.linspace(0, 1, 40)
    y = np.linspace(0, 2, 50)
    A = 1.0 / (1.0 + (x[:, None] - y[None, :]) ** 2)
    rf, cf, r1, c1 = _matrix_fns(A)
    blk = cross.aca_block(rf, cf, 40, 50, 1e-8, 40, b)
    rep = cross.aca(r1, c1, 40, 50, 1e-8, 40, pivots=list(zip(blk["I"], blk["J"])))
    scale = np.abs(A).max()
    assert np.max(np.abs(blk["U"] @ blk["V"].T - rep["U"] @ rep["V"].T)) <= 1e-12 * scale
    a, ia = cross.htaca(fn, N, 1e-8, 16, return_info=True, block=b)
    r, ir = cross.htaca(fn, N, 1e-8, 16, pivots=ia["pivots"], return_info=True)
    assert np.allclose(_dense(a), _dense(r), atol=1e-12 * np.abs(_dense(a)).max())


@pytest.mark.parametrize("b", [2, 4])
def test_block_htaca_of_sl_update_close_to_dense(b):
    """SLAR with blocks: within 10 eps of the dense SL step on a tiny 2D-2V grid, and the
    first SLAR call of 2D-2V weak Landau 32^4 within eps of the dense update (the case the
    rank-1 test alone missed by 84 eps)."""
    N = (10, 10, 12, 12)
    g = sl.PhaseGrid(2, 2, N, (0, 0, -5, -5), (4 * math.pi, 4 * math.pi, 5, 5))
    w = inputs.landau_2d2v(n=10, alpha=0.3)
    w.N, w.lo, w.hi = N, g.lo, g.hi
    F0 = htmod.truncate(htmod.from_terms(inputs.initial_factors(w)), 1e-12, 20)
    E = inputs.random_field(N[:2], 2, 0.3, seed=2)
    eps = 1e-6
    out = cross.htaca(lambda idx: sl.sl_eval(F0, E, 0.4, idx, g), N, eps, 40, block=b)
    dense = sl.dense_sl_step(htmod.densify(F0), E, 0.4, g)
    assert np.linalg.norm(_dense(out) - dense) <= 10 * eps * np.linalg.norm(dense)
