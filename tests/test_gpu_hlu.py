"""The block LU of the reflection matrix on the GPU (§5.1) and its forward and
backward substitution (§5.2), against the oracle's H-LU (oracle/hlu.py) and
the dense direct solve: without truncation it is the unique LU of C; with
truncation at eps_rel its error follows eps_rel as the oracle's does; as a
right preconditioner it cuts the GMRES iterations without changing the
solution."""
import numpy as np
import pytest

import cavities as cv
from gpu_common import rad
from oracle import SIGMA_SB, geometry, hlu, viewfactor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cube():
    verts = cv.unit_cube(6)                                   # 432 facets
    f = geometry.facets_from_triangles(verts)
    F = viewfactor.dense(f)
    eps = np.random.default_rng(8).uniform(0.3, 0.9, f.size)
    C = np.eye(f.size) - (1.0 - eps)[:, None] * F
    r = rad()
    h = r.rad_build_htree(verts, 16, 1.0)
    # F stored to ~1e-13 (full pivoting, Eq. 31 exactly): C is the oracle's C
    r.rad_compress_aca(h, 1e-13, 64, "full", "f64", "f64")
    perm = r.rad_htree_export_tree(h)["perm"]
    yield dict(verts=verts, f=f, F=F, eps=eps, C=C, h=h, perm=perm)
    h.free()


def _split(LU):
    return np.tril(LU, -1) + np.eye(LU.shape[0]), np.triu(LU)


def test_without_truncation_it_is_the_unique_lu_of_c(cube):
    r = rad()
    lu = r.rad_hlu_factor(cube["h"], cube["eps"], 0.0)
    st = r.rad_hlu_get_stats(lu)
    assert st["n_lowrank"] == 0 and st["precision"] == r.RAD_F64
    Lg, Ug = _split(r.rad_hlu_export(lu))
    o = hlu.factor(cube["F"], cube["eps"], cube["f"].c, 16, 1.0, 0.0)
    assert np.array_equal(o.perm, cube["perm"])                # same tree (Algorithm 1)
    Lo, Uo = o.factors()
    assert np.linalg.norm(Lg - Lo) <= 1e-11 * np.linalg.norm(Lo)
    assert np.linalg.norm(Ug - Uo) <= 1e-11 * np.linalg.norm(Uo)
    b = np.random.default_rng(1).uniform(size=(cube["C"].shape[0], 3))
    x = r.rad_hlu_solve(lu, b)
    xe = np.linalg.solve(cube["C"], b)
    assert np.linalg.norm(x - xe) <= 1e-11 * np.linalg.norm(xe)
    lu.free()


@pytest.mark.parametrize("tol", [1e-3, 1e-5])
def test_truncated_factors_follow_eps_rel_like_the_oracle(cube, tol):
    r = rad()
    C, perm = cube["C"], cube["perm"]
    Ct = C[np.ix_(perm, perm)]
    lu = r.rad_hlu_factor(cube["h"], cube["eps"], tol)
    st = r.rad_hlu_get_stats(lu)
    Lg, Ug = _split(r.rad_hlu_export(lu))
    err_gpu = np.linalg.norm(Lg @ Ug - Ct) / np.linalg.norm(Ct)
    o = hlu.factor(cube["F"], cube["eps"], cube["f"].c, 16, 1.0, tol)
    Lo, Uo = o.factors()
    err_oracle = np.linalg.norm(Lo @ Uo - Ct) / np.linalg.norm(Ct)
    # the pin the oracle meets, and the same order of error as the oracle
    assert err_gpu <= 10 * tol, err_gpu
    assert err_oracle <= 10 * tol
    assert err_gpu <= 3 * err_oracle + 1e-3 * tol, (err_gpu, err_oracle)
    # compression: never more entries than the dense LU; at 1e-3 the
    # admissible leaves of this small cube are stored low rank (at 1e-5 most
    # need more terms than their storage break-even rank and stay dense)
    assert st["dense_entries"] + st["lowrank_entries"] <= C.size
    if tol >= 1e-3:
        assert st["n_lowrank"] > 0 and st["dense_entries"] + st["lowrank_entries"] < C.size
    # solve error within the conditioning of C, and close to the oracle's H-LU solve
    kappa = np.linalg.cond(C)
    b = np.random.default_rng(2).uniform(size=C.shape[0])
    x = r.rad_hlu_solve(lu, b)
    xe = np.linalg.solve(C, b)
    assert np.linalg.norm(x - xe) <= 10 * kappa * tol * np.linalg.norm(xe)
    xo = o.solve_blocks(b)
    assert np.linalg.norm(x - xo) <= 20 * kappa * tol * np.linalg.norm(xe)
    lu.free()


def test_fp32_factors_on_a_cylinder():
    r = rad()
    verts = cv.closed_cylinder(1.0, 4.0, 40, 24, 4)           # 2,480 facets
    f = geometry.facets_from_triangles(verts)
    F = viewfactor.dense(f)
    eps = np.random.default_rng(3).uniform(0.3, 0.9, f.size)
    C = np.eye(f.size) - (1.0 - eps)[:, None] * F
    h = r.rad_build_htree(verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "f32", "f32")
    tol = 1e-4
    lu = r.rad_hlu_factor(h, eps, tol)
    st = r.rad_hlu_get_stats(lu)
    assert st["precision"] == r.RAD_F32 and st["n_lowrank"] > 0
    perm = r.rad_htree_export_tree(h)["perm"]
    Lg, Ug = _split(r.rad_hlu_export(lu))
    Ct = C[np.ix_(perm, perm)]
    assert np.linalg.norm(Lg @ Ug - Ct) / np.linalg.norm(Ct) <= 10 * tol
    b = np.random.default_rng(4).uniform(size=(f.size, 2))
    x = r.rad_hlu_solve(lu, b)
    xe = np.linalg.solve(C, b)
    assert np.linalg.norm(x - xe) <= 10 * np.linalg.cond(C) * tol * np.linalg.norm(xe)
    lu.free()
    h.free()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_preconditioned_gmres_converges_in_fewer_iterations_to_the_same_flux(dtype):
    r = rad()
    c = cv.config1()                                         # 768 facets
    T = np.asfortranarray(c.T[:, :1] * np.array([1.0, 0.8, 1.2]))
    h = r.rad_build_htree(c.verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-8 if dtype == "f64" else 1e-6, 64, "partial", dtype, dtype)
    stol = 1e-10 if dtype == "f64" else 1e-6          # FP32 storage: residuals to ~1e-7
    q0, i0 = r.rad_solve_flux(h, c.eps, T, SIGMA_SB, tol=stol)
    lu = r.rad_hlu_factor(h, c.eps, 1e-4)
    q1, i1 = r.rad_solve_flux(h, c.eps, T, SIGMA_SB, tol=stol, precond=lu)
    assert i0["status"] == 0 and i1["status"] == 0
    assert i1["iters"] <= max(3, i0["iters"] // 3), (i0["iters"], i1["iters"])
    tolq = 1e-8 if dtype == "f64" else 1e-5
    assert np.linalg.norm(q1 - q0) <= tolq * np.linalg.norm(q0)
    # factors of other emissivities still precondition (the test is on C itself)
    lu2 = r.rad_hlu_factor(h, np.full(c.n, 0.5), 1e-4)
    q2, i2 = r.rad_solve_flux(h, c.eps, T, SIGMA_SB, tol=stol, precond=lu2)
    assert i2["status"] == 0 and np.linalg.norm(q2 - q0) <= tolq * np.linalg.norm(q0)
    lu.free()
    lu2.free()
    h.free()


def test_batch_handle_factors_every_cavity():
    r = rad()
    cavs = [cv.config1()] + [cv.Cavity("cube4", cv.unit_cube(4), np.full(192, 0.6),
                                       np.full((192, 1), 900.0), {})]
    counts = [c.n for c in cavs]
    verts = np.concatenate([c.verts for c in cavs])
    eps = np.concatenate([c.eps for c in cavs])
    h = r.rad_build_htree_batch(verts, counts, 32, 1.0)
    r.rad_compress_aca(h, 1e-8, 64, "partial", "f64", "f64")
    lu = r.rad_hlu_factor(h, eps, 1e-6)
    b = np.random.default_rng(5).uniform(size=sum(counts))
    x = r.rad_hlu_solve(lu, b)
    off = 0
    for c in cavs:
        F = viewfactor.dense(geometry.facets_from_triangles(c.verts))
        C = np.eye(c.n) - (1.0 - eps[off:off + c.n])[:, None] * F
        xe = np.linalg.solve(C, b[off:off + c.n])
        assert np.linalg.norm(x[off:off + c.n] - xe) <= 1e-4 * np.linalg.norm(xe)
        off += c.n
    lu.free()
    h.free()


def test_invalid_arguments():
    r = rad()
    c = cv.config1()
    h = r.rad_build_htree(c.verts, 32, 1.0)
    with pytest.raises(r.RadError):
        r.rad_hlu_factor(h, c.eps, 1e-4)                     # not compressed
    r.rad_compress_aca(h, 1e-6, 64, "partial", "f64", "f64")
    e = c.eps.copy()
    e[3] = 1.5
    with pytest.raises(r.RadError) as ex:
        r.rad_hlu_factor(h, e, 1e-4)
    assert ex.value.code == r.RAD_EINVAL
    with pytest.raises(r.RadError):
        r.rad_hlu_factor(h, c.eps, -1.0)
    h2 = r.rad_build_htree(c.verts, 32, 1.0)
    r.rad_compress_aca(h2, 1e-6, 64, "partial", "f64", "f64")
    lu2 = r.rad_hlu_factor(h2, c.eps, 1e-4)
    with pytest.raises(r.RadError) as ex:                    # factors of another handle
        r.rad_solve_flux(h, c.eps, c.T, SIGMA_SB, tol=1e-8, precond=lu2)
    assert ex.value.code == r.RAD_EINVAL
    lu2.free()
    h2.free()
    h.free()
