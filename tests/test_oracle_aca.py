"""Pins for the oracle's cross approximation (§4.3, Eqs. 30-31)."""
import math

import numpy as np
import pytest

import cavities as cv
from oracle import aca, geometry, htree, viewfactor


def _rank_r(m, n, r, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, r)) @ rng.standard_normal((r, n))


@pytest.mark.parametrize("m,n,r", [(30, 20, 1), (40, 55, 4), (64, 64, 9)])
def test_full_pivot_recovers_exact_rank(m, n, r):
    X = _rank_r(m, n, r, m + n)
    U, V, ok, R, C = aca.aca_full(X, 1e-12, 50)
    assert ok and U.shape[1] == r
    assert np.linalg.norm(X - U @ V.T) <= 1e-12 * np.linalg.norm(X) * 10


@pytest.mark.parametrize("m,n,r", [(30, 20, 1), (40, 55, 4), (64, 64, 9)])
def test_partial_pivot_recovers_exact_rank(m, n, r):
    X = _rank_r(m, n, r, 3 * m + n)
    U, V, ok = aca.aca_partial(lambda i: X[i], lambda j: X[:, j], m, n, 1e-12, 50)
    assert ok and U.shape[1] >= r
    assert np.linalg.norm(X - U @ V.T) <= 1e-10 * np.linalg.norm(X)


def test_full_pivot_is_the_cross_of_eq30():
    """U V^T equals X(:,C) X(R,C)^-1 X(R,:) for the chosen pivots."""
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, 50)
    y = rng.uniform(3, 4, 40)
    X = 1.0 / (x[:, None] - y[None, :]) ** 2            # smooth, numerically low rank
    U, V, ok, R, C = aca.aca_full(X, 1e-8, 40)
    k = U.shape[1]
    assert ok and 2 <= k < 20
    cross = X[:, C] @ np.linalg.solve(X[np.ix_(R, C)], X[R, :])
    assert np.linalg.norm(cross - U @ V.T) <= 1e-9 * np.linalg.norm(X)
    # Eq. (31) holds, and one rank fewer would not have satisfied it
    assert np.linalg.norm(X - U @ V.T) <= 1e-8 * np.linalg.norm(X)
    Uk, Vk = U[:, :-1], V[:, :-1]
    assert np.linalg.norm(X - Uk @ Vk.T) > 1e-8 * np.linalg.norm(X)
    # the pivot rows/columns are distinct and the pivots are reproduced
    assert len(set(R)) == k and len(set(C)) == k
    np.testing.assert_allclose((U @ V.T)[np.ix_(R, C)], X[np.ix_(R, C)], rtol=1e-10)


def test_partial_pivot_meets_tolerance_on_view_factor_blocks():
    f = geometry.facets_from_triangles(cv.closed_cylinder(1.0, 4.0, 40, 24, 4))
    t = htree.build_cluster_tree(f.c, 24)
    ft = f.subset(t.perm)
    blocks = [b for b in htree.build_block_tree(t, 1.0) if b.admissible]
    rng = np.random.default_rng(1)
    for k in rng.choice(len(blocks), 25, replace=False):
        b = blocks[k]
        rows = np.arange(b.row.begin, b.row.end)
        cols = np.arange(b.col.begin, b.col.end)
        X = viewfactor.rows(ft, rows, cols)
        U, V, ok = aca.aca_partial(lambda i: X[i], lambda j: X[:, j], len(rows), len(cols), 1e-6, 64)
        assert ok
        if np.linalg.norm(X) > 0:
            # the partial-pivot stopping rule is an estimate: allow 10x slack
            assert np.linalg.norm(X - U @ V.T) <= 1e-5 * np.linalg.norm(X)
            s = np.linalg.svd(X, compute_uv=False)
            need = int((np.sqrt(np.cumsum(s[::-1] ** 2))[::-1] > 1e-6 * np.linalg.norm(X)).sum())
            assert U.shape[1] <= 2 * need + 3


def test_zero_block_has_rank_zero_and_sphere_block_rank_one():
    X = np.zeros((20, 30))
    U, V, ok = aca.aca_partial(lambda i: X[i], lambda j: X[:, j], 20, 30, 1e-6, 10)
    assert ok and U.shape[1] == 0
    U, V, ok, _, _ = aca.aca_full(X, 1e-6, 10)
    assert ok and U.shape[1] == 0
    # sphere identity: every row of F is A_j / (4 pi R^2) -> rank one
    rng = np.random.default_rng(5)
    p = rng.normal(size=(60, 3))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    f = geometry.Facets(p, -p, rng.uniform(0.01, 0.02, 60))
    X = viewfactor.rows(f, np.arange(0, 30), np.arange(30, 60))
    U, V, ok = aca.aca_partial(lambda i: X[i], lambda j: X[:, j], 30, 30, 1e-10, 10)
    assert ok and U.shape[1] == 1
    assert np.linalg.norm(X - U @ V.T) <= 1e-13 * np.linalg.norm(X)


def test_rank_cap_reports_not_converged():
    X = np.random.default_rng(0).standard_normal((20, 20))
    U, V, ok = aca.aca_partial(lambda i: X[i], lambda j: X[:, j], 20, 20, 1e-12, 5)
    assert not ok and U.shape[1] == 5
    U, V, ok, _, _ = aca.aca_full(X, 1e-12, 5)
    assert not ok


def test_partial_norm_estimate_is_exact_frobenius_of_the_cross():
    """The running ||S_k||_F^2 with all cross terms equals ||U V^T||_F^2."""
    rng = np.random.default_rng(11)
    x = rng.uniform(0, 1, 45)
    y = rng.uniform(2, 3, 35)
    X = 1.0 / (x[:, None] - y[None, :]) ** 2
    st = {}
    U, V, ok = aca.aca_partial(lambda i: X[i], lambda j: X[:, j], 45, 35, 1e-10, 30, stats=st)
    assert ok and U.shape[1] >= 3
    exact = float(np.linalg.norm(U @ V.T) ** 2)
    assert abs(st["norm2_S"] - exact) <= 1e-12 * exact
    assert st["rows"][0] == 0


def test_plain_partial_pivot_can_stop_early_where_full_pivot_meets_eq31():
    """§1 calls partial pivoting less reliable than full pivoting.  A block
    of a box cavity (1 x 4.85 x 3.26, 28,336 facets) shows it: the plain
    partial-pivot stop fires with about 9% of the block unapproximated,
    because the pivots never visit the rows that carry it, while full
    pivoting on the same block meets Eq. (31) exactly."""
    f = geometry.facets_from_triangles(cv.box(1.0, 4.845306857887991, 3.2594759571933496, 17, 84, 56))
    t = htree.build_cluster_tree(f.c, 64)
    perm = np.asarray(t.perm)
    X = viewfactor.rows(f, perm[21252:21694], perm[3099:3542])
    m, n = X.shape
    tol = 1e-6
    U, V, ok = aca.aca_partial(lambda i: X[i], lambda j: X[:, j], m, n, tol, 64)
    assert ok and np.linalg.norm(X - U @ V.T) / np.linalg.norm(X) > 1e-2
    U, V, ok, _, _ = aca.aca_full(X, tol, 64)
    assert ok and np.linalg.norm(X - U @ V.T) <= tol * np.linalg.norm(X)


def test_truncation_keeps_the_product_within_tolerance_and_drops_redundant_rank():
    """Rank truncation (§4.3 standard form, §5.1 relative accuracy): an
    exact rank-3 product written with 7 redundant terms comes back at rank
    3 to rounding; a numerically low-rank cross is cut to the rank the
    singular-value decay allows, within tol."""
    rng = np.random.default_rng(4)
    A, B = rng.normal(size=(40, 3)), rng.normal(size=(30, 3))
    C = rng.normal(size=(3, 7))
    U, V = A @ C, B @ np.linalg.pinv(C).T          # U V^T = A B^T, 7 terms
    Ut, Vt = aca.truncate(U, V, 1e-10)
    assert Ut.shape[1] == 3
    assert np.linalg.norm(Ut @ Vt.T - A @ B.T) <= 1e-12 * np.linalg.norm(A @ B.T)
    x = np.linspace(0.0, 1.0, 60)
    y = np.linspace(2.0, 3.0, 50)
    X = 1.0 / (x[:, None] - y[None, :]) ** 2
    U, V, ok = aca.aca_partial(lambda i: X[i], lambda j: X[:, j], 60, 50, 1e-12, 40)
    for tol in (1e-4, 1e-7):
        Ut, Vt = aca.truncate(U, V, tol)
        s = np.linalg.svd(X, compute_uv=False)
        # the exact optimal rank for tol, give or take the ACA error
        r_opt = next(r for r in range(1, len(s) + 1) if np.sqrt((s[r:] ** 2).sum()) <= tol * np.linalg.norm(s))
        assert abs(Ut.shape[1] - r_opt) <= 1
        assert np.linalg.norm(X - Ut @ Vt.T) <= 1.01 * tol * np.linalg.norm(X) + 1e-11 * np.linalg.norm(X)
    assert aca.truncate(np.zeros((5, 2)), np.zeros((4, 2)), 1e-6)[0].shape[1] == 0
