"""Pins for the oracle's hierarchical LU of the reflection matrix (§5.1) and
its substitutions (§5.2): without truncation it is the (unique) LU
factorisation of C; with truncation at eps_rel its error follows eps_rel and
it stores fewer entries than without truncation; a closed cavity solves to
z = 1."""
import numpy as np
import pytest

import cavities as cv
from oracle import geometry, hlu, viewfactor


@pytest.fixture(scope="module")
def cube():
    f = geometry.facets_from_triangles(cv.unit_cube(6))     # 432 facets
    F = viewfactor.dense(f)
    eps = np.random.default_rng(8).uniform(0.3, 0.9, f.size)
    C = np.eye(f.size) - (1.0 - eps)[:, None] * F
    return f, F, eps, C


def test_without_truncation_it_is_the_lu_of_c(cube):
    f, F, eps, C = cube
    h = hlu.factor(F, eps, f.c, n_min=16, eta=1.0, tol=0.0)
    L, U = h.factors()
    Ct = C[np.ix_(h.perm, h.perm)]
    # unit lower times upper triangular reproduces C: the LU without
    # pivoting, which is unique
    assert np.array_equal(np.triu(L, 1), np.zeros_like(L)) and np.allclose(np.diag(L), 1.0)
    assert np.array_equal(np.tril(U, -1), np.zeros_like(U))
    assert np.linalg.norm(L @ U - Ct) <= 1e-13 * np.linalg.norm(Ct)
    b = np.random.default_rng(1).uniform(size=f.size)
    x = h.solve(b)
    assert np.linalg.norm(x - np.linalg.solve(C, b)) <= 1e-12 * np.linalg.norm(x)


@pytest.mark.parametrize("tol", [1e-3, 1e-5, 1e-7])
def test_truncation_error_follows_eps_rel(cube, tol):
    f, F, eps, C = cube
    h = hlu.factor(F, eps, f.c, n_min=16, eta=1.0, tol=tol)
    L, U = h.factors()
    Ct = C[np.ix_(h.perm, h.perm)]
    rel = np.linalg.norm(L @ U - Ct) / np.linalg.norm(Ct)
    # every block the factorisation produces and every admissible block of C is truncated
    # at tol relative to itself; over the few levels of this tree the
    # factorisation error stays within a small multiple of tol
    assert rel <= 10 * tol, rel
    b = np.random.default_rng(2).uniform(size=f.size)
    x = h.solve(b)
    xe = np.linalg.solve(C, b)
    kappa = np.linalg.cond(C)
    assert np.linalg.norm(x - xe) <= 10 * kappa * tol * np.linalg.norm(xe)
    # the truncation is applied: fewer stored entries than without it
    exact = hlu.factor(F, eps, f.c, n_min=16, eta=1.0, tol=0.0)
    assert h.stored_entries() < exact.stored_entries()


def test_error_decreases_with_eps_rel(cube):
    f, F, eps, C = cube
    errs = []
    for tol in (1e-2, 1e-4, 1e-6):
        h = hlu.factor(F, eps, f.c, n_min=16, eta=1.0, tol=tol)
        L, U = h.factors()
        Ct = C[np.ix_(h.perm, h.perm)]
        errs.append(np.linalg.norm(L @ U - Ct) / np.linalg.norm(Ct))
    assert errs[0] > errs[1] > errs[2]


def test_closed_cavity_solves_to_one():
    """Unit row sums give C 1 = eps (closed cavity), so the H-LU solve of
    C z = eps returns z = 1; the admissible blocks of (J - I)/(n - 1) are
    rank one, so truncation loses nothing."""
    f = geometry.facets_from_triangles(cv.unit_cube(4))      # 192 facets
    n = f.size
    F = (np.ones((n, n)) - np.eye(n)) / (n - 1)
    eps = np.random.default_rng(3).uniform(0.2, 0.9, n)
    h = hlu.factor(F, eps, f.c, n_min=16, eta=1.0, tol=1e-8)
    np.testing.assert_allclose(h.solve(eps), 1.0, rtol=1e-10)


def test_truncation_keeps_the_smallest_admissible_rank():
    """truncate_dense: the kept rank is the smallest with the dropped
    singular values below tol ||M||_F, and the result is the SVD truncation."""
    rng = np.random.default_rng(4)
    W, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    Z, _ = np.linalg.qr(rng.standard_normal((20, 20)))
    s = 10.0 ** -np.arange(20)
    M = (W[:, :20] * s) @ Z.T
    total = np.sqrt((s * s).sum())
    for tol, r in ((2e-3, 3), (5e-7, 7), (0.0, 20)):
        U, V = hlu.truncate_dense(M, tol)
        assert U.shape[1] == r, (tol, U.shape[1])
        assert np.linalg.norm(M - U @ V.T) <= tol * total * (1 + 1e-9) + 1e-14


@pytest.mark.parametrize("tol", [0.0, 1e-5])
def test_block_substitution_equals_dense_substitution(cube, tol):
    """§5.2: forward and backward substitution through the block structure
    (low-rank blocks applied as U (V^T x)) add no approximation: they equal
    the dense triangular solves with the same factors."""
    f, F, eps, C = cube
    h = hlu.factor(F, eps, f.c, n_min=16, eta=1.0, tol=tol)
    b = np.random.default_rng(6).uniform(size=f.size)
    x_dense = h.solve(b)
    x_blocks = h.solve_blocks(b)
    assert np.linalg.norm(x_blocks - x_dense) <= 1e-12 * np.linalg.norm(x_dense)
