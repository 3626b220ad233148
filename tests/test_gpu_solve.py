"""GPU GMRES reflection solve (Eq. 11) and flux (Eq. 12) against closed
forms and the oracle's direct solve."""
import numpy as np
import pytest

import cavities as cv
from gpu_common import rad, rel
from oracle import SIGMA_SB, geometry, radiosity, viewfactor

pytestmark = pytest.mark.gpu


def test_two_grey_planes_eq5():
    r = rad()
    h = r.rad_htree_from_dense(np.array([[0.0, 1.0], [1.0, 0.0]]))
    for e1, e2, T1, T2 in [(0.3, 0.8, 400.0, 900.0), (0.9, 0.1, 1200.0, 300.0)]:
        q, info = r.rad_solve_flux(h, np.array([e1, e2]), np.array([T1, T2]), SIGMA_SB, tol=1e-14)
        want = radiosity.two_planes_flux(e2, e1, T2, T1, SIGMA_SB)
        assert abs(q[0] - want) <= 1e-12 * abs(want)
        assert abs(q[1] + want) <= 1e-12 * abs(want)


def test_closed_cavity_and_uniform_temperature():
    r = rad()
    n = 9
    F = (np.ones((n, n)) - np.eye(n)) / (n - 1)
    h = r.rad_htree_from_dense(F)
    eps = np.linspace(0.2, 0.9, n)
    Y, info = r.rad_solve_reflection(h, eps, eps, tol=1e-14)
    np.testing.assert_allclose(Y, 1.0, rtol=1e-12)
    q, _ = r.rad_solve_flux(h, eps, np.full(n, 500.0), SIGMA_SB, tol=1e-14)
    assert np.abs(q).max() <= 1e-12 * SIGMA_SB * 500.0 ** 4


def test_c1_fp64_flux_within_1e6_and_conserves_energy():
    c = cv.config1()
    f = geometry.facets_from_triangles(c.verts)
    F = viewfactor.dense(f)
    q_ref, _, _ = radiosity.solve_flux(F, c.eps, c.T, SIGMA_SB)
    r = rad()
    h = r.rad_build_htree(c.verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "f64", "f64")
    q, info = r.rad_solve_flux(h, c.eps, c.T, SIGMA_SB, tol=1e-12)
    assert info["status"] == 0
    assert rel(q, q_ref) <= 1e-6
    assert abs((f.area * q[:, 0]).sum()) <= 1e-6 * (f.area * np.abs(q[:, 0])).sum()


def test_multi_field_fp64_and_fp32():
    verts = cv.closed_cylinder(1.0, 4.0, 40, 24, 4)
    f = geometry.facets_from_triangles(verts)
    F = viewfactor.dense(f)
    rng = np.random.default_rng(9)
    eps = rng.uniform(0.3, 0.9, f.size)
    T = rng.uniform(300, 1200, (f.size, 5))
    q_ref, Y_ref, z_ref = radiosity.solve_flux(F, eps, T, SIGMA_SB)
    r = rad()
    h = r.rad_build_htree(verts, 24, 1.0)
    r.rad_compress_aca(h, 1e-9, 64, "partial", "f64", "f64")
    q, info = r.rad_solve_flux(h, eps, T, SIGMA_SB, tol=1e-12)
    for c in range(5):
        assert rel(q[:, c], q_ref[:, c]) <= 1e-6
    B = np.concatenate([eps[:, None] * T ** 4, eps[:, None]], axis=1)
    Y, info = r.rad_solve_reflection(h, eps, B, tol=1e-12)
    assert rel(Y[:, :5], Y_ref) <= 1e-8 and rel(Y[:, 5], z_ref) <= 1e-8
    r.rad_compress_aca(h, 1e-8, 64, "partial", "f32", "f32")
    q32, info = r.rad_solve_flux(h, eps, T, SIGMA_SB, tol=1e-7)
    assert rel(q32, q_ref) <= 1e-5


def test_not_converged_is_reported():
    c = cv.config1()
    r = rad()
    h = r.rad_build_htree(c.verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "f64", "f64")
    q, info = r.rad_solve_flux(h, c.eps, c.T, SIGMA_SB, tol=1e-14, max_iter=2)
    assert info["status"] == r.RAD_ENOTCONV
    assert info["iters"] == 2
    with pytest.raises(r.RadError):
        r.rad_solve_flux(h, c.eps, c.T, SIGMA_SB, tol=1e-14, max_iter=2, raise_on_notconv=True)


def test_device_buffers_equal_host_buffers():
    import torch
    c = cv.config1()
    r = rad()
    h = r.rad_build_htree(c.verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "f64", "f64")
    qh, _ = r.rad_solve_flux(h, c.eps, c.T, SIGMA_SB, tol=1e-12)
    qd, _ = r.rad_solve_flux(h, torch.as_tensor(c.eps, device="cuda"), torch.as_tensor(c.T, device="cuda"),
                             SIGMA_SB, tol=1e-12)
    np.testing.assert_array_equal(qd.cpu().numpy(), qh)


def _sphere_facets(n=400, seed=8, fill=0.8, R=1.5):
    rng = np.random.default_rng(seed)
    p = rng.normal(size=(n, 3))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    area = rng.uniform(0.5, 1.5, size=n)
    area *= fill * 4.0 * np.pi * R * R / area.sum()
    return geometry.Facets(R * p, -p, area)


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
def test_closed_cavity_rows_match_the_oracle(dt):
    """§6 closed cavity: after rad_htree_close_cavity the stored operator is
    the oracle's row-scaled F (facets on a sphere, where s_i is known in
    closed form), and its rows sum to 1."""
    f = _sphere_facets()
    r = rad()
    h = r.rad_build_htree_facets(f.c, f.n, f.area, leaf_size=16, eta_adm=1.0)
    near = "f64" if dt == "f64" else "f32"
    r.rad_compress_aca(h, 1e-10 if dt == "f64" else 1e-6, 64, "partial", dt, near,
                       accurate_dtype=None if dt != "bf16" else "f32")
    s = r.rad_htree_close_cavity(h)
    F = viewfactor.dense(f)
    Fc, s_ref, _ = radiosity.close_cavity(F)
    assert r.rad_htree_get_stats(h)["closed"] == 1
    assert np.abs(s - s_ref).max() <= (1e-9 if dt == "f64" else 2e-6)
    x = np.random.default_rng(3).uniform(0.5, 1.5, f.c.shape[0])
    xin = x if dt == "f64" else x.astype(np.float32)
    tol = {"f64": 1e-9, "f32": 2e-6, "bf16": 1e-2}[dt]
    assert rel(r.rad_hmatvec(h, xin), Fc @ x) <= tol
    ones = np.ones(f.c.shape[0]) if dt == "f64" else np.ones(f.c.shape[0], np.float32)
    assert np.abs(r.rad_hmatvec(h, ones) - 1.0).max() <= tol
    h.free()


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_one_column_reflection_solve_in_fp32_storage_meets_the_direct_solve(dt):
    """One right-hand side on an FP32 or BF16 operator (the one-column
    product inside GMRES reads the FP32 copy of each Krylov vector), alone
    and in a batch of two cavities, against the oracle's direct solve of
    Eq. (11)."""
    c = cv.config1()
    f = geometry.facets_from_triangles(c.verts)
    F = viewfactor.dense(f)
    b = SIGMA_SB * c.eps * c.T[:, 0] ** 4
    y_ref = np.linalg.solve(radiosity.reflection_matrix(F, c.eps), b)
    r = rad()
    h = r.rad_build_htree(c.verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-7, 64, "partial", dt, "f32", accurate_dtype="f32" if dt == "bf16" else None)
    kw = dict(refine=True, inner_tol=1e-4, tol=1e-8) if dt == "bf16" else dict(tol=1e-7)
    y, info = r.rad_solve_reflection(h, c.eps, b, **kw)
    assert info["status"] == 0
    assert rel(y, y_ref) <= 1e-6
    h.free()
    hb = r.rad_build_htree_batch(np.concatenate([c.verts, c.verts]), [c.n, c.n], 32, 1.0)
    r.rad_compress_aca(hb, 1e-7, 64, "partial", dt, "f32", accurate_dtype="f32" if dt == "bf16" else None)
    yb, info = r.rad_solve_reflection(hb, np.concatenate([c.eps, c.eps]), np.concatenate([b, 2 * b]), **kw)
    assert info["status"] == 0
    assert rel(yb[:c.n], y_ref) <= 1e-6 and rel(yb[c.n:], 2 * y_ref) <= 1e-6
    hb.free()
