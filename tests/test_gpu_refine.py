"""Mixed precision with iterative refinement: BF16 low-rank factors for the
GMRES corrections, an FP32 copy with FP64 accumulation for the residuals."""
import numpy as np
import pytest

import cavities as cv
from gpu_common import rad, rel
from oracle import SIGMA_SB, geometry, radiosity, viewfactor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    verts = cv.closed_cylinder(1.0, 4.0, 40, 24, 4)
    f = geometry.facets_from_triangles(verts)
    F = viewfactor.dense(f)
    rng = np.random.default_rng(21)
    eps = rng.uniform(0.1, 0.95, f.size)
    T = rng.uniform(300, 1200, (f.size, 2))
    q_ref, _, _ = radiosity.solve_flux(F, eps, T, SIGMA_SB)
    return verts, F, eps, T, q_ref


def test_refined_bf16_matches_oracle_and_plain_bf16_does_not(case):
    verts, F, eps, T, q_ref = case
    r = rad()
    h = r.rad_build_htree(verts, 24, 1.0)
    r.rad_compress_aca(h, 1e-7, 64, "partial", "bf16", "f32", accurate_dtype="f32")
    st = r.rad_htree_get_stats(h)
    assert st["bytes_accurate"] > 0
    q_plain, info_plain = r.rad_solve_flux(h, eps, T, SIGMA_SB, tol=1e-6)
    q, info = r.rad_solve_flux(h, eps, T, SIGMA_SB, tol=1e-9, refine=True, inner_tol=1e-4)
    assert info["status"] == 0 and info["refinements"] >= 1
    assert info["max_rel_residual"] <= 1e-9
    assert rel(q, q_ref) <= 1e-6
    assert rel(q_plain, q_ref) > 1e-5          # BF16 alone is not accurate enough


def test_refined_solution_matches_the_fp64_operator(case):
    verts, F, eps, T, q_ref = case
    r = rad()
    h64 = r.rad_build_htree(verts, 24, 1.0)
    r.rad_compress_aca(h64, 1e-7, 64, "partial", "f64", "f64")
    B = np.concatenate([eps[:, None] * T ** 4, eps[:, None]], axis=1)
    Y64, _ = r.rad_solve_reflection(h64, eps, B, tol=1e-12)
    hm = r.rad_build_htree(verts, 24, 1.0)
    r.rad_compress_aca(hm, 1e-7, 64, "partial", "bf16", "f32", accurate_dtype="f32")
    Y, info = r.rad_solve_reflection(hm, eps, B, tol=1e-10, refine=True, inner_tol=1e-4)
    assert info["status"] == 0
    # same ACA factors (FP64 ACA arithmetic at this tolerance), FP32-rounded
    for c in range(B.shape[1]):
        assert rel(Y[:, c], Y64[:, c]) <= 1e-6


def test_refinement_needs_an_accurate_operator(case):
    verts, F, eps, T, q_ref = case
    r = rad()
    h = r.rad_build_htree(verts, 24, 1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "bf16", "f32")
    with pytest.raises(r.RadError) as ei:
        r.rad_solve_flux(h, eps, T, SIGMA_SB, tol=1e-9, refine=True)
    assert ei.value.code == r.RAD_EINVAL
