"""GPU dense-block entries (Eq. 10) and ACA (Eqs. 30-31) against the oracle's
FP64 entries, block by block."""
import math

import numpy as np
import pytest

import cavities as cv
from gpu_common import dense_tree_order, gpu_blocks, rad
from oracle import geometry

pytestmark = pytest.mark.gpu


def _check_blocks(h, Ft, tol, near_rtol, far_slack, exact_full=False):
    r = rad()
    tr, bl, keys = gpu_blocks(h)
    worst = 0.0
    n_lr = 0
    for b, (r0, r1, c0, c1, adm) in enumerate(keys):
        X = Ft[r0:r1, c0:c1]
        rk = int(bl["rank"][b])
        if rk < 0:
            D = r.rad_htree_export_block(h, b, r1 - r0, c1 - c0, rk)
            np.testing.assert_allclose(D, X, rtol=near_rtol, atol=near_rtol * max(np.abs(X).max(), 1e-300))
            continue
        assert adm
        U, V = r.rad_htree_export_block(h, b, r1 - r0, c1 - c0, rk)
        nx = np.linalg.norm(X)
        err = np.linalg.norm(X - U @ V.T)
        if nx == 0:
            assert rk == 0
            continue
        n_lr += 1
        worst = max(worst, err / nx)
        if exact_full:
            assert err <= tol * nx * (1 + 1e-6) + 1e-15 * nx, (b, err / nx)
        else:
            assert err <= far_slack * tol * nx, (b, err / nx)
    return worst, n_lr


def test_fp64_partial_blocks_cylinder():
    r = rad()
    verts = cv.closed_cylinder(1.0, 4.0, 48, 30, 4)
    h = r.rad_build_htree(verts, 24, 1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "f64", "f64")
    tr = r.rad_htree_export_tree(h)
    _, Ft = dense_tree_order(verts, tr["perm"])
    worst, n_lr = _check_blocks(h, Ft, 1e-6, 1e-13, 10.0)
    assert n_lr > 10


def test_fp64_full_pivot_meets_eq31_exactly():
    r = rad()
    verts = cv.closed_cylinder(1.0, 4.0, 32, 20, 3)
    h = r.rad_build_htree(verts, 16, 1.0)
    r.rad_compress_aca(h, 1e-5, 64, "full", "f64", "f64")
    tr = r.rad_htree_export_tree(h)
    _, Ft = dense_tree_order(verts, tr["perm"])
    worst, n_lr = _check_blocks(h, Ft, 1e-5, 1e-13, 1.0, exact_full=True)
    assert n_lr > 10


def test_fp32_blocks():
    r = rad()
    verts = cv.closed_cylinder(1.0, 4.0, 48, 30, 4)
    h = r.rad_build_htree(verts, 24, 1.0)
    r.rad_compress_aca(h, 1e-5, 64, "partial", "f32", "f32")
    tr = r.rad_htree_export_tree(h)
    _, Ft = dense_tree_order(verts, tr["perm"])
    _check_blocks(h, Ft, 1e-5, 2e-6, 10.0)


def test_cube_coplanar_blocks_are_rank_zero():
    r = rad()
    c = cv.config1()
    h = r.rad_build_htree(c.verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "f64", "f64")
    tr = r.rad_htree_export_tree(h)
    _, Ft = dense_tree_order(c.verts, tr["perm"])
    _, bl, keys = gpu_blocks(h)
    for b, (r0, r1, c0, c1, adm) in enumerate(keys):
        if adm and not Ft[r0:r1, c0:c1].any():
            assert bl["rank"][b] == 0
    _check_blocks(h, Ft, 1e-6, 1e-13, 10.0)


def test_sphere_identity_blocks_have_rank_one():
    """Facets on a sphere with radial normals: F_ij = A_j / (4 pi R^2), so
    every admissible block is exactly rank one."""
    r = rad()
    rng = np.random.default_rng(3)
    p = rng.normal(size=(600, 3))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    area = rng.uniform(0.001, 0.002, 600)
    h = r.rad_build_htree_facets(2.0 * p, -p, area, 16, 1.0)
    r.rad_compress_aca(h, 1e-10, 64, "partial", "f64", "f64")
    _, bl, keys = gpu_blocks(h)
    adm = bl["admissible"] == 1
    assert adm.sum() > 0
    assert (bl["rank"][adm] == 1).all()
    U, V = None, None
    for b, (r0, r1, c0, c1, a) in enumerate(keys):
        if a:
            U, V = r.rad_htree_export_block(h, b, r1 - r0, c1 - c0, 1)
            perm = r.rad_htree_export_tree(h)["perm"]
            X = np.broadcast_to(area[perm[c0:c1]] / (16.0 * math.pi), (r1 - r0, c1 - c0))
            np.testing.assert_allclose(U @ V.T, X, rtol=1e-12)
            break


def test_rank_cap_falls_back_to_dense():
    r = rad()
    verts = cv.closed_cylinder(1.0, 4.0, 32, 20, 3)
    h = r.rad_build_htree(verts, 16, 1.0)
    r.rad_compress_aca(h, 1e-12, 1, "partial", "f64", "f64")
    st = r.rad_htree_get_stats(h)
    assert st["n_dense_fallback"] > 0
    tr = r.rad_htree_export_tree(h)
    _, Ft = dense_tree_order(verts, tr["perm"])
    _check_blocks(h, Ft, 1e-12, 1e-13, 10.0)


def test_bad_parameters_rejected():
    r = rad()
    h = r.rad_build_htree(cv.unit_cube(2), 4, 1.0)
    with pytest.raises(r.RadError):
        r.rad_compress_aca(h, 1e-6, 64, "partial", "f64", "f32")
    with pytest.raises(r.RadError):
        r.rad_compress_aca(h, -1.0, 64, "partial", "f64", "f64")
    with pytest.raises(r.RadError):
        r.rad_hmatvec(h, np.ones(h.n))           # not compressed yet
