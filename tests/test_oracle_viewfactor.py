"""Pins for the oracle's geometry and view-factor entries (Eq. 10, §3.2).

Every check here is fixed by geometry or by a closed form, not by re-running
the oracle's own formula.
"""
import math
import os

import numpy as np
import pytest

import cavities as cv
from oracle import geometry, viewfactor

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_plates():
    out = {}
    for line in open(os.path.join(GOLDEN, "plates_closed_form.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, val, tol = line.split()
        out[name] = (float(val), float(tol))
    return out


def parallel_squares_exact(X, Y):
    """Aligned parallel rectangles a x b at distance c, X = a/c, Y = b/c."""
    return 2.0 / (math.pi * X * Y) * (
        0.5 * math.log((1 + X * X) * (1 + Y * Y) / (1 + X * X + Y * Y))
        + X * math.sqrt(1 + Y * Y) * math.atan(X / math.sqrt(1 + Y * Y))
        + Y * math.sqrt(1 + X * X) * math.atan(Y / math.sqrt(1 + X * X))
        - X * math.atan(X) - Y * math.atan(Y))


def perpendicular_exact(W, H):
    """Perpendicular rectangles with a common edge of length l, W = w/l, H = h/l."""
    s = math.sqrt(H * H + W * W)
    a = (1 + W * W) * (1 + H * H) / (1 + W * W + H * H)
    b = (W * W * (1 + W * W + H * H) / ((1 + W * W) * (W * W + H * H))) ** (W * W)
    c = (H * H * (1 + H * H + W * W) / ((1 + H * H) * (H * H + W * W))) ** (H * H)
    return (W * math.atan(1 / W) + H * math.atan(1 / H) - s * math.atan(1 / s)
            + 0.25 * math.log(a * b * c)) / (math.pi * W)


def test_triangle_geometry_hand_values():
    v = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0]],
                  [[0, 0, 2], [0, 3, 2], [4, 0, 2]]], dtype=float)
    f = geometry.facets_from_triangles(v)
    np.testing.assert_allclose(f.c[0], [1 / 3, 1 / 3, 0], rtol=0, atol=1e-16)
    np.testing.assert_allclose(f.n[0], [0, 0, 1])
    assert f.area[0] == 0.5
    np.testing.assert_allclose(f.c[1], [4 / 3, 1.0, 2.0], atol=1e-15)
    np.testing.assert_allclose(f.n[1], [0, 0, -1])
    assert f.area[1] == 6.0


def test_mesh_areas_and_inward_normals():
    f = geometry.facets_from_triangles(cv.unit_cube(8))
    assert f.size == 768
    np.testing.assert_allclose(f.area, 1.0 / 128.0, rtol=1e-14)
    inward = np.einsum("ij,ij->i", f.n, np.array([0.5, 0.5, 0.5]) - f.c)
    assert (inward > 0).all()
    v = cv.closed_cylinder()
    f = geometry.facets_from_triangles(v)
    assert f.size == 19936
    ns = 112
    side = ns * 2 * math.sin(math.pi / ns) * 4.0
    caps = 2 * ns * 0.5 * math.sin(2 * math.pi / ns)
    assert abs(f.area.sum() - (side + caps)) < 1e-10
    radial = f.c[:, :2]
    side_mask = (f.c[:, 2] > 1e-9) & (f.c[:, 2] < 4 - 1e-9)
    assert (np.einsum("ij,ij->i", f.n[side_mask, :2], -radial[side_mask]) > 0).all()
    assert (f.n[f.c[:, 2] < 1e-12, 2] > 0.999).all()
    assert (f.n[f.c[:, 2] > 4 - 1e-12, 2] < -0.999).all()
    s = geometry.facets_from_triangles(cv.icosphere(3))
    assert s.size == 20 * 4 ** 3
    assert (np.einsum("ij,ij->i", s.n, -s.c) > 0).all()


def test_plate_closed_forms_match_handbook_values():
    g = _golden_plates()
    val, tol = g["parallel_coaxial_unit_gap_1"]
    assert abs(parallel_squares_exact(1.0, 1.0) - val) < tol
    val, tol = g["perpendicular_common_edge"]
    assert abs(perpendicular_exact(1.0, 1.0) - val) < tol
    # a cube face sees the opposite face and four adjacent faces: sum = 1
    total = parallel_squares_exact(1.0, 1.0) + 4.0 * perpendicular_exact(1.0, 1.0)
    assert abs(total - 1.0) < 1e-12


def test_parallel_plates_converge_second_order():
    exact = parallel_squares_exact(1.0, 1.0)
    errs = []
    for n in (4, 8, 16):
        v = cv.parallel_plates(1.0, n, 1.0)
        errs.append(viewfactor.plate_to_plate(v, 2 * n * n) - exact)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, errs
    # Richardson extrapolation (h^2) lands on the closed form
    rich = (4 * (errs[2] + exact) - (errs[1] + exact)) / 3
    assert abs(rich - exact) < 2e-6


def test_perpendicular_plates_converge_first_order():
    exact = perpendicular_exact(1.0, 1.0)
    vals = []
    for n in (8, 16, 32):
        v = cv.perpendicular_plates(1.0, n)
        vals.append(viewfactor.plate_to_plate(v, 2 * n * n))
    errs = [x - exact for x in vals]
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2, errs
    rich = 2 * vals[2] - vals[1]
    assert abs(rich - exact) < 5e-5


def test_sphere_identity():
    """Facets on a sphere with inward radial normals: F_ij = A_j / (4 pi R^2)."""
    rng = np.random.default_rng(7)
    R = 2.5
    p = rng.normal(size=(40, 3))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    area = rng.uniform(0.01, 0.1, size=40)
    f = geometry.Facets(R * p, -p, area)
    F = viewfactor.dense(f)
    expect = np.broadcast_to(area / (4 * math.pi * R * R), F.shape).copy()
    np.fill_diagonal(expect, 0.0)
    np.testing.assert_allclose(F, expect, rtol=1e-12, atol=0)


def test_zero_diagonal_reciprocity_and_backfacing():
    f = geometry.facets_from_triangles(cv.closed_cylinder(1.0, 4.0, 24, 12, 3))
    F = viewfactor.dense(f)
    assert (np.diag(F) == 0).all()
    AF = f.area[:, None] * F
    np.testing.assert_allclose(AF, AF.T, rtol=1e-12, atol=1e-300)
    # two facets that face away from each other exchange nothing
    g = geometry.Facets(np.array([[0, 0, 0], [0, 0, 1.0]]),
                        np.array([[0, 0, -1.0], [0, 0, 1.0]]), np.array([1.0, 1.0]))
    assert (viewfactor.dense(g) == 0).all()


def test_scalar_entry_agrees_with_vectorised_rows():
    f = geometry.facets_from_triangles(cv.unit_cube(3))
    F = viewfactor.dense(f)
    for i in range(0, f.size, 7):
        for j in range(0, f.size, 5):
            e = 0.0 if i == j else viewfactor.entry(f.c[i], f.n[i], f.c[j], f.n[j], f.area[j])
            assert abs(e - F[i, j]) <= 1e-15 * max(1.0, abs(e))


def test_centroid_rule_within_composite_quadrature_spread():
    """For well separated facets the 1-point rule sits within the composite
    rule's convergence range (brute-force quadrature of Eq. 10)."""
    v = cv.parallel_plates(1.0, 2, 1.0)
    f = geometry.facets_from_triangles(v)
    rows = [0, 3]
    cols = [8, 12]
    c0 = viewfactor.rows(f, rows, cols)
    seq = [viewfactor.composite(v, L, rows, cols) for L in (0, 1, 2, 3)]
    np.testing.assert_allclose(seq[0], c0, rtol=1e-13)
    # composite sequence converges (Cauchy) and the centroid rule error is
    # of the size of the first refinement step
    d23 = np.abs(seq[3] - seq[2])
    d12 = np.abs(seq[2] - seq[1])
    assert (d23 < 0.35 * d12 + 1e-15).all()
    assert (np.abs(c0 - seq[3]) <= 2.0 * np.abs(seq[1] - seq[0]) + 1e-15).all()


def test_cube_row_sums_tend_to_one():
    """Enclosure rule: sum_j F_ij -> 1 as the closed cube is refined."""
    worst = []
    for n in (2, 4, 8):
        f = geometry.facets_from_triangles(cv.unit_cube(n))
        F = viewfactor.dense(f)
        worst.append(np.abs(F.sum(axis=1) - 1.0).max())
    assert worst[0] > worst[1] > worst[2]
    # area-weighted mean row sum is much closer to one than the worst row
    f = geometry.facets_from_triangles(cv.unit_cube(8))
    F = viewfactor.dense(f)
    mean = float((f.area * F.sum(axis=1)).sum() / f.area.sum())
    assert abs(mean - 1.0) < 0.05
