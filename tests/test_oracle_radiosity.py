"""Pins for the oracle's reflection solve and facet flux (Eqs. 5, 11, 12) and
for its hierarchical matrix (§4-5)."""
import math

import numpy as np
import pytest

import cavities as cv
from oracle import SIGMA_SB, geometry, hmatrix, radiosity, viewfactor


def test_two_grey_planes_eq5():
    """Two facets that see only each other reproduce the infinite-plane
    formula of Eq. (5) (flux into facet 1 = flux from 2 to 1)."""
    F = np.array([[0.0, 1.0], [1.0, 0.0]])
    for e1, e2, T1, T2 in [(0.3, 0.8, 400.0, 900.0), (0.9, 0.1, 1200.0, 300.0), (1.0, 1.0, 500.0, 600.0)]:
        q, _, _ = radiosity.solve_flux(F, np.array([e1, e2]), np.array([T1, T2]), SIGMA_SB)
        want = radiosity.two_planes_flux(e2, e1, T2, T1, SIGMA_SB)
        assert abs(q[0] - want) <= 1e-13 * abs(want)
        assert abs(q[1] + want) <= 1e-13 * abs(want)


def test_closed_cavity_z_is_one():
    """Unit row sums (closed cavity): C 1 = eps, so z = C^-1 eps = 1."""
    n = 9
    F = (np.ones((n, n)) - np.eye(n)) / (n - 1)
    eps = np.linspace(0.2, 0.9, n)
    _, _, z = radiosity.solve_flux(F, eps, np.full(n, 500.0), SIGMA_SB)
    np.testing.assert_allclose(z, 1.0, rtol=1e-14)


def test_uniform_temperature_gives_zero_flux():
    f = geometry.facets_from_triangles(cv.unit_cube(4))
    F = viewfactor.dense(f)
    eps = np.random.default_rng(2).uniform(0.3, 0.9, f.size)
    q, Y, z = radiosity.solve_flux(F, eps, np.full(f.size, 800.0), SIGMA_SB)
    scale = SIGMA_SB * 800.0 ** 4
    assert np.abs(q).max() <= 1e-12 * scale


def test_energy_conservation():
    """sum_i A_i q_i = 0 whenever A_i F_ij = A_j F_ji (R is symmetric, Eq. 17)."""
    c = cv.config1()
    f = geometry.facets_from_triangles(c.verts)
    F = viewfactor.dense(f)
    q, _, _ = radiosity.solve_flux(F, c.eps, c.T[:, 0], SIGMA_SB)
    assert abs((f.area * q).sum()) <= 1e-12 * (f.area * np.abs(q)).sum()
    # and R = sigma eps_i eps_j (F C^-1)_ij scaled by A_i is symmetric
    C = radiosity.reflection_matrix(F, c.eps)
    R = SIGMA_SB * c.eps[:, None] * c.eps[None, :] * (F @ np.linalg.inv(C))
    AR = f.area[:, None] * R
    np.testing.assert_allclose(AR, AR.T, rtol=1e-9, atol=1e-12 * np.abs(AR).max())


def test_flux_matches_eq12_written_with_the_papers_matrix():
    """Eq. (12) evaluated literally with F_paper = diag(A) F and Lambda = (1-eps)/A."""
    f = geometry.facets_from_triangles(cv.unit_cube(2))
    F = viewfactor.dense(f)
    A = f.area
    rng = np.random.default_rng(4)
    eps = rng.uniform(0.3, 0.9, f.size)
    T = rng.uniform(300, 1200, f.size)
    eta = T ** 4
    Fp = A[:, None] * F
    Cp = np.eye(f.size) - ((1 - eps) / A)[:, None] * Fp
    Cinv = np.linalg.inv(Cp)
    q_lit = np.zeros(f.size)
    for i in range(f.size):
        s = 0.0
        for j in range(f.size):
            s += eps[j] * (Fp[i, :] @ Cinv[:, j]) * (eta[j] - eta[i])
        q_lit[i] = SIGMA_SB * eps[i] / A[i] * s
    q, _, _ = radiosity.solve_flux(F, eps, T, SIGMA_SB)
    np.testing.assert_allclose(q, q_lit, rtol=1e-10, atol=1e-10 * np.abs(q_lit).max())


def test_hmatrix_exact_when_tolerance_vanishes():
    f = geometry.facets_from_triangles(cv.closed_cylinder(1.0, 4.0, 24, 16, 3))
    F = viewfactor.dense(f)
    x = np.random.default_rng(0).uniform(size=f.size)
    H = hmatrix.build(f, 16, 1.0, 0.0, "full", max_rank=10 ** 6)
    assert np.linalg.norm(H.matvec(x) - F @ x) <= 1e-13 * np.linalg.norm(F @ x)
    np.testing.assert_allclose(H.to_dense(), F, rtol=0, atol=1e-15)


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6])
def test_hmatrix_error_bounded_by_tolerance(tol):
    """Eq. (31) per block (full pivoting, exact) => ||F - F_eps||_F <= eps ||F||_F."""
    f = geometry.facets_from_triangles(cv.closed_cylinder(1.0, 4.0, 32, 20, 4))
    F = viewfactor.dense(f)
    H = hmatrix.build(f, 16, 1.0, tol, "full")
    err = np.linalg.norm(H.to_dense() - F) / np.linalg.norm(F)
    assert err <= tol
    assert any(b.rank > 0 for b in H.leaves)


def test_sampled_rows_agree_with_dense():
    c = cv.config1()
    f = geometry.facets_from_triangles(c.verts)
    F = viewfactor.dense(f)
    rows = np.array([0, 5, 300, 767])
    x = c.T[:, 0] ** 4
    np.testing.assert_allclose(radiosity.matvec_rows(f, rows, x), (F @ x)[rows], rtol=1e-13)
    np.testing.assert_allclose(radiosity.rowsum_rows(f, rows), F.sum(axis=1)[rows], rtol=1e-13)


def test_closed_cavity_rows_follow_the_clamp_rule():
    """§6 closed cavity: rows with 0 < s_i <= 1 sum to 1 after the scaling,
    rows with s_i > 1 or s_i = 0 are left alone (c_i = 1 or c_i = 0)."""
    rng = np.random.default_rng(2)
    F = rng.uniform(0.0, 0.2, (6, 6))
    F[1] *= 10.0           # s > 1: c = 1, row kept
    F[2] = 0.0             # s = 0: c = 0, row kept
    Fc, s, c = radiosity.close_cavity(F)
    assert s[1] > 1.0 and c[1] == 1.0 and np.array_equal(Fc[1], F[1])
    assert s[2] == 0.0 and c[2] == 0.0 and np.array_equal(Fc[2], F[2])
    for i in (0, 3, 4, 5):
        assert 0.0 < s[i] <= 1.0
        assert abs(Fc[i].sum() - 1.0) <= 1e-15
        np.testing.assert_allclose(Fc[i], F[i] / s[i], rtol=1e-15)
    # facets on a sphere with inward radial normals: F_ij = A_j / (4 pi R^2)
    # (sphere identity), so s_i = (A - A_i) / (4 pi R^2) with A = sum of areas;
    # with A below the sphere's area every row is scaled to sum 1, and row i
    # becomes A_j / (A - A_i)
    rng = np.random.default_rng(8)
    R = 1.5
    p = rng.normal(size=(60, 3))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    area = rng.uniform(0.5, 1.5, size=60)
    area *= 0.8 * 4.0 * math.pi * R * R / area.sum()
    f = geometry.Facets(R * p, -p, area)
    Fc, s, c = radiosity.close_cavity(viewfactor.dense(f))
    np.testing.assert_allclose(s, (area.sum() - area) / (4.0 * math.pi * R * R), rtol=1e-12)
    expect = area[None, :] / (area.sum() - area)[:, None]
    np.fill_diagonal(expect, 0.0)
    np.testing.assert_allclose(Fc, expect, rtol=1e-12)
