"""GPU block low-rank matvec (§5.2) against the oracle's dense F x."""
import numpy as np
import pytest

import cavities as cv
from gpu_common import rad, rel
from oracle import SIGMA_SB, geometry, viewfactor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    c = cv.config1()
    f = geometry.facets_from_triangles(c.verts)
    return c, viewfactor.dense(f)


@pytest.fixture(scope="module")
def cyl():
    verts = cv.closed_cylinder(1.0, 4.0, 56, 36, 5)     # 4,592 facets
    f = geometry.facets_from_triangles(verts)
    return verts, viewfactor.dense(f)


def test_c1_fp64_matvec_within_1e6(c1):
    c, F = c1
    r = rad()
    h = r.rad_build_htree(c.verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "f64", "f64")
    x = SIGMA_SB * c.T[:, 0] ** 4
    y = r.rad_hmatvec(h, x)
    assert rel(y, F @ x) <= 1e-6


def test_fp64_exact_when_tolerance_vanishes(cyl):
    verts, F = cyl
    r = rad()
    h = r.rad_build_htree(verts, 32, 1.0)
    r.rad_compress_aca(h, 0.0, 128, "full", "f64", "f64")
    x = np.random.default_rng(0).uniform(size=F.shape[0])
    assert rel(r.rad_hmatvec(h, x), F @ x) <= 1e-12


@pytest.mark.parametrize("nrhs", [1, 2, 3, 4, 17, 65, 130])
def test_multi_rhs_fp64_and_fp32(cyl, nrhs):
    verts, F = cyl
    r = rad()
    X = np.random.default_rng(nrhs).uniform(0.5, 1.5, size=(F.shape[0], nrhs))
    Yref = F @ X
    h = r.rad_build_htree(verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-9, 64, "partial", "f64", "f64")
    Y = r.rad_hmatvec(h, X)
    for c in range(nrhs):
        assert rel(Y[:, c], Yref[:, c]) <= 1e-7, c
    r.rad_compress_aca(h, 1e-8, 64, "partial", "f32", "f32")
    Y32 = r.rad_hmatvec(h, X.astype(np.float32))
    for c in range(nrhs):
        assert rel(Y32[:, c], Yref[:, c]) <= 1e-6, c


def test_bf16_factors(cyl):
    verts, F = cyl
    r = rad()
    h = r.rad_build_htree(verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "bf16", "f32")
    x = np.random.default_rng(1).uniform(0.5, 1.5, size=F.shape[0]).astype(np.float32)
    e = rel(r.rad_hmatvec(h, x), F @ x)
    assert e <= 1e-2


def test_device_strided_and_host_paths_agree(cyl):
    import torch
    verts, F = cyl
    r = rad()
    h = r.rad_build_htree(verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-7, 64, "partial", "f32", "f32")
    n = F.shape[0]
    X = np.random.default_rng(2).uniform(size=(n, 5))
    Yh = r.rad_hmatvec(h, X)
    big = torch.zeros((5, n + 7), dtype=torch.float64, device="cuda")
    big[:, :n] = torch.as_tensor(X.T, device="cuda")
    Xd = big.t()[:n]                                     # column-major view, ld = n + 7
    Yd = r.rad_hmatvec(h, Xd)
    np.testing.assert_array_equal(Yd.cpu().numpy(), Yh)


def test_caller_provided_outputs(c1):
    import torch
    c, F = c1
    r = rad()
    h = r.rad_build_htree(c.verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "f32", "f32")
    x = torch.as_tensor(c.T[:, 0], device="cuda", dtype=torch.float32)
    y = torch.empty_like(x)
    out = r.rad_hmatvec(h, x, y)
    assert out.data_ptr() == y.data_ptr()
    assert rel(y.cpu().numpy(), F @ c.T[:, 0]) <= 1e-6


@pytest.mark.parametrize("factor", ["f32", "bf16"])
@pytest.mark.parametrize("path", [0, 1])
def test_many_column_paths_match_column_by_column(cyl, factor, path):
    """The many-column product, on CUDA cores (path 0) and on tensor cores
    (path 1, BF16 x 3 split), equals the one-column streaming product column
    by column to FP32 accuracy, for FP32 and BF16 factors (same stored
    operator)."""
    verts, F = cyl
    r = rad()
    h = r.rad_build_htree(verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", factor, "f32")
    r.rad_htree_set_product_path(h, path)
    assert r.rad_htree_get_stats(h)["product_path"] == path
    X = np.random.default_rng(7).uniform(-1.0, 1.5, size=(F.shape[0], 9)).astype(np.float32)
    Y = r.rad_hmatvec(h, X)
    for c in range(9):
        y1 = r.rad_hmatvec(h, np.ascontiguousarray(X[:, c]))
        # FP32 rounding of sums of |F| |x|: scale by the product with |x|
        scale = np.abs(r.rad_hmatvec(h, np.ascontiguousarray(np.abs(X[:, c])))).max()
        assert np.abs(Y[:, c] - y1).max() <= 2e-6 * scale, c


@pytest.mark.parametrize("nc", [5, 9, 64, 65, 96, 130])
def test_tensor_core_product_against_the_dense_oracle(cyl, nc):
    """The tensor-core product (path 1) against the oracle's dense F X, column
    by column, beside the CUDA-core product (path 0): both within the FP32
    bound of the operator (ACA tol 1e-7) and within FP32 rounding of each
    other (a few FP32 ulps).  Covers one and two column chunks (96 per launch) and ragged
    widths (N padded to a multiple of 8)."""
    verts, F = cyl
    r = rad()
    h = r.rad_build_htree(verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-7, 64, "partial", "f32", "f32")
    X = np.random.default_rng(nc).uniform(0.0, 1.0, size=(F.shape[0], nc)).astype(np.float32)
    ref = F @ X.astype(np.float64)
    out = {}
    for path in (0, 1):
        r.rad_htree_set_product_path(h, path)
        out[path] = r.rad_hmatvec(h, X).astype(np.float64)
        for c in range(nc):
            assert rel(out[path][:, c], ref[:, c]) <= 1e-6, (path, c)
    # the two paths round differently (FFMA sums whole panels in FP32, the
    # tensor cores restart every 128 columns): FP32-level agreement
    assert np.abs(out[1] - out[0]).max() <= 5e-6 * np.abs(ref).max()
    r.rad_htree_free(h)


def test_tensor_core_path_in_the_solver_meets_the_oracle():
    """The flux solve with the tensor-core product (every GMRES product and
    the flux epilogue) against the oracle's direct solve."""
    r = rad()
    verts = cv.closed_cylinder(1.0, 4.0, 40, 24, 4)
    rng = np.random.default_rng(6)
    eps = rng.uniform(0.3, 0.9, verts.shape[0])
    T = rng.uniform(300, 1200, (verts.shape[0], 12))
    F = viewfactor.dense(geometry.facets_from_triangles(verts))
    from oracle import radiosity
    qref, _, _ = radiosity.solve_flux(F, eps, T, SIGMA_SB)
    h = r.rad_build_htree(verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-7, 64, "partial", "f32", "f32")
    q0, i0 = r.rad_solve_flux(h, eps, T, SIGMA_SB, tol=1e-7)
    r.rad_htree_set_product_path(h, 1)
    q1, i1 = r.rad_solve_flux(h, eps, T, SIGMA_SB, tol=1e-7)
    assert i0["status"] == 0 and i1["status"] == 0
    for q in (q0, q1):
        assert rel(q, qref) <= 1e-6
    r.rad_htree_free(h)


@pytest.mark.parametrize("factor", ["f32", "bf16"])
def test_one_column_fused_and_two_launch_paths_against_the_oracle(cyl, factor):
    """The one-column product in one fused launch (bulk-copy ring, A units
    then B units) and in two launches: both within the FP32 bound of F x,
    agreeing with each other to rounding, on a cavity whose column groups
    span several 16 KiB stages and whose index slices start off 16-byte
    boundaries."""
    verts, F = cyl
    r = rad()
    x = np.random.default_rng(5).uniform(0.5, 1.5, size=F.shape[0])
    yref = F @ x
    h = r.rad_build_htree(verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-8, 64, "partial", factor, "f32")
    assert r.rad_htree_get_stats(h)["one_column_path"] == 1
    y1 = r.rad_hmatvec(h, x.astype(np.float32))
    r.rad_htree_set_one_column_path(h, 0)
    assert r.rad_htree_get_stats(h)["one_column_path"] == 0
    y0 = r.rad_hmatvec(h, x.astype(np.float32))
    bound = 1e-6 if factor == "f32" else 5e-3
    assert rel(y1, yref) <= bound and rel(y0, yref) <= bound
    assert rel(y1, y0) <= 2e-6
    # repeated launches: the same bits (fixed summation order per row)
    r.rad_htree_set_one_column_path(h, 1)
    for _ in range(3):
        np.testing.assert_array_equal(r.rad_hmatvec(h, x.astype(np.float32)), y1)
    h.free()


def test_one_column_fused_path_in_the_solver_and_after_closing(c1):
    """The fused launch with the reflection epilogues of Eq. (11) inside
    GMRES, and on a closed cavity (rows rescaled in place)."""
    c, F = c1
    r = rad()
    h = r.rad_build_htree(c.verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-7, 64, "partial", "f32", "f32")
    assert r.rad_htree_get_stats(h)["one_column_path"] == 1
    T = np.asfortranarray(c.T[:, :1])
    q1, i1 = r.rad_solve_flux(h, c.eps, T, SIGMA_SB, tol=1e-7)
    r.rad_htree_set_one_column_path(h, 0)
    q0, i0 = r.rad_solve_flux(h, c.eps, T, SIGMA_SB, tol=1e-7)
    assert i1["status"] == 0 and i0["status"] == 0
    assert rel(q1, q0) <= 1e-6
    r.rad_htree_set_one_column_path(h, 1)
    s = r.rad_htree_close_cavity(h)
    y = r.rad_hmatvec(h, np.ones(h.n, dtype=np.float32))
    expect = np.where((s > 0) & (s <= 1), 1.0, s)   # rows divided by clamp(s, 0, 1)
    np.testing.assert_allclose(y, expect, rtol=0, atol=2e-6)
    h.free()
