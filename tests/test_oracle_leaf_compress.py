"""Oracle pins: leaf bases of rank r_mu from the cross factors (``cross.compress_leaves``,
step 2' of the HTACA reading) in place of identity leaves of order N_mu, and the greedy
column-pivoted QR (``cross.qrcp_basis``) that chooses them.

* qrcp_basis: every greedy choice is the column of largest residual norm, recomputed here by
  explicit projection; the returned basis is orthonormal, its residual is at most the
  tolerance and one column fewer would not have been; on an exactly rank-3 matrix it stops
  at 3 columns spanning the SVD's range; ties go to the lowest index.
* compress_leaves: on an HT of exact leaf ranks (3, 2, 4, 3) with unequal N (a transposed
  unfolding would give other ranks) the leaf ranks are recovered exactly and the tensor to
  rounding; on smooth data the error is within the first-order bound 4 eps_l ||A||_F,
  eps_l = eps / (2 sqrt 5), with leaves of rank below N -- also from factors rescaled by a
  diagonal D and D^-1 (the same A), which the weighting by the other side's triangular
  factor makes irrelevant.
* htaca with leaf_compress: within 10 eps of the dense SL step (as the identity-leaf path)
  and within 2 eps of the identity-leaf result.
"""
import math

import numpy as np
import pytest

from oracle import cross, sl
from oracle import ht as htmod
from paper_2606_29027_b300 import inputs


def _resid(M, Q):
    return float(np.linalg.norm(M - Q @ (Q.T @ M)))


def test_qrcp_greedy_choices_by_projection():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((7, 9)) @ np.diag(np.linspace(3.0, 0.2, 9))
    Q, cols = cross.qrcp_basis(M, 1e-12 * np.linalg.norm(M))
    assert len(cols) == 7 and len(set(cols)) == 7
    for t, j in enumerate(cols):
        P = Q[:, :t]
        R = M - P @ (P.T @ M)
        norms = np.linalg.norm(R, axis=0)
        norms[cols[:t]] = -1.0
        assert j == int(np.argmax(norms))
    assert np.allclose(Q.T @ Q, np.eye(7), atol=1e-13)


@pytest.mark.parametrize("rel", [0.5, 0.1, 1e-2, 1e-4])
def test_qrcp_stops_at_the_first_column_count_within_tolerance(rel):
    rng = np.random.default_rng(5)
    M = (rng.standard_normal((20, 6)) @ rng.standard_normal((6, 30))
         + 1e-3 * rng.standard_normal((20, 30)))
    tol = rel * np.linalg.norm(M)
    Q, cols = cross.qrcp_basis(M, tol)
    assert np.allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-12)
    assert _resid(M, Q) <= tol * (1 + 1e-12)
    if Q.shape[1] > 0:
        assert _resid(M, Q[:, :-1]) > tol


def test_qrcp_exact_rank_spans_svd_range():
    rng = np.random.default_rng(7)
    M = rng.standard_normal((15, 3)) @ rng.standard_normal((3, 11))
    Q, cols = cross.qrcp_basis(M, 1e-12 * np.linalg.norm(M))
    assert Q.shape[1] == 3
    Us = np.linalg.svd(M)[0][:, :3]
    # principal angles between the two 3-dimensional subspaces: all cosines 1
    assert np.allclose(np.linalg.svd(Us.T @ Q, compute_uv=False), 1.0, atol=1e-10)


def test_qrcp_tie_goes_to_the_lowest_index():
    M = np.array([[1.0, 0.0, 3.0, 0.0], [0.0, 2.0, 0.0, 3.0]])
    _, cols = cross.qrcp_basis(M, 0.0)
    assert cols[0] == 2   # columns 2 and 3 both have norm 3
    assert cols[1] == 3


def _root_factors(F, N):
    M1 = int(np.prod(N[:2]))
    A = F.reshape(M1, -1)
    Us, s, Vt = np.linalg.svd(A, full_matrices=False)
    k = int(np.count_nonzero(s > 1e-13 * s[0]))
    return Us[:, :k] * s[:k], Vt[:k].T, A


def test_compress_leaves_recovers_exact_leaf_ranks():
    N = (8, 9, 7, 10)
    h = htmod.from_raw(inputs.random_ht(N, (3, 2, 4, 3, 4, 5), 12, smooth=False))
    F = htmod.densify(h)
    U, V, A = _root_factors(F, N)
    c = cross.compress_leaves(U, V, N, 1e-12)
    assert [u.shape[1] for u in c.U] == [3, 2, 4, 3]
    for u in c.U:
        assert np.allclose(u.T @ u, np.eye(u.shape[1]), atol=1e-13)
    assert np.linalg.norm(htmod.densify(c) - F) <= 1e-11 * np.linalg.norm(F)


@pytest.mark.parametrize("rescale", [False, True])
@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-6])
def test_compress_leaves_error_within_first_order_bound(eps, rescale):
    N = (10, 12, 11, 9)
    x1 = np.linspace(0, 2 * np.pi, N[0], endpoint=False)
    x2 = np.linspace(0, 2 * np.pi, N[1], endpoint=False)
    v1 = np.linspace(-4, 4, N[2])
    v2 = np.linspace(-4, 4, N[3])
    X1, X2, V1, V2 = np.meshgrid(x1, x2, v1, v2, indexing="ij")
    F = (1 + 0.3 * np.cos(X1) * np.cos(2 * X2)) * np.exp(-0.5 * (V1 ** 2 + V2 ** 2)) \
        + 0.2 * np.sin(X1 + X2) * np.exp(-0.5 * ((V1 - 1) ** 2 + (V2 + 0.5) ** 2) / 0.7)
    U, V, A = _root_factors(F, N)
    if rescale:   # the same A from factors of very different column scales (A = U D (V D^-1)^T)
        D = np.logspace(-3, 3, U.shape[1])
        U, V = U * D, V / D
    c = cross.compress_leaves(U, V, N, eps)
    eps_l = eps / (2 * math.sqrt(5))
    err = np.linalg.norm(htmod.densify(c).reshape(A.shape) - A)
    assert err <= 4 * eps_l * np.linalg.norm(A) * (1 + 1e-9)
    if eps >= 1e-4:
        assert all(u.shape[1] < n for u, n in zip(c.U, N))


def test_htaca_leaf_compress_close_to_dense_and_to_identity_leaves():
    N = (10, 10, 12, 12)
    g = sl.PhaseGrid(2, 2, N, (0, 0, -5, -5), (4 * math.pi, 4 * math.pi, 5, 5))
    w = inputs.landau_2d2v(n=10, alpha=0.3)
    w.N, w.lo, w.hi = N, g.lo, g.hi
    F0 = htmod.truncate(htmod.from_terms(inputs.initial_factors(w)), 1e-12, 20)
    E = inputs.random_field(N[:2], 2, 0.3, seed=2)
    eps = 1e-6
    fn = lambda idx: sl.sl_eval(F0, E, 0.4, idx, g)
    ident, ii = cross.htaca(fn, N, eps, 40, return_info=True)
    comp, ic = cross.htaca(fn, N, eps, 40, return_info=True, leaf_compress=True, pivots=ii["pivots"])
    dense = sl.dense_sl_step(htmod.densify(F0), E, 0.4, g)
    nd = np.linalg.norm(dense)
    assert np.linalg.norm(htmod.densify(comp) - dense) <= 10 * eps * nd
    assert np.linalg.norm(htmod.densify(comp) - htmod.densify(ident)) <= 2 * eps * nd
    assert all(abs(a - b) <= 1 for a, b in zip(ic["ranks"], ii["ranks"]))
