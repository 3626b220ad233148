"""Full-size parity on sampled rows: the cylinder of the benchmark (19,936
facets, 64 fields, FP32) and the level-6 icosphere (81,920 facets, BF16
factors with FP64-residual refinement).  The oracle evaluates the sampled
rows of F exactly (centroid rule) one by one; solves are checked through
exact residual rows of Eq. (11)."""
import numpy as np
import pytest

import cavities as cv
from gpu_common import rad
from oracle import SIGMA_SB, geometry, radiosity

pytestmark = pytest.mark.gpu


def _sample(n, k=512, seed=0):
    return np.sort(np.random.default_rng(seed).choice(n, k, replace=False))


def test_cylinder_bench_configuration_sampled_rows():
    import torch
    c = cv.config2(m=64)
    r = rad()
    h = r.rad_build_htree(torch.as_tensor(c.verts, device="cuda"), 64, 1.0)
    r.rad_compress_aca(h, 1e-5, 64, "partial", "f32", "f32")
    f = geometry.facets_from_triangles(c.verts)
    rows = _sample(c.n)
    X = SIGMA_SB * c.T ** 4
    Y = r.rad_hmatvec(h, torch.as_tensor(X, device="cuda", dtype=torch.float32)).cpu().numpy()
    ref = radiosity.matvec_rows(f, rows, X)
    assert np.linalg.norm(Y[rows] - ref) / np.linalg.norm(ref) <= 2e-6
    # the reflection solve of the bench (tol 1e-7) through exact residual rows
    B = np.concatenate([c.eps[:, None] * c.T ** 4, c.eps[:, None]], axis=1)
    Ys, info = r.rad_solve_reflection(h, c.eps, B, tol=1e-7)
    assert info["status"] == 0
    res = radiosity.residual_rows(f, c.eps, rows, Ys, B)
    assert np.linalg.norm(res) / np.linalg.norm(B[rows]) <= 2e-6


@pytest.mark.slow
def test_icosphere6_mixed_precision_sampled_rows():
    import torch
    c = cv.config3()
    r = rad()
    h = r.rad_build_htree(torch.as_tensor(c.verts, device="cuda"), 64, 1.0)
    r.rad_compress_aca(h, 1e-7, 64, "partial", "bf16", "f32", accurate_dtype="f32")
    f = geometry.facets_from_triangles(c.verts)
    rows = _sample(c.n, seed=3)
    B = np.concatenate([c.eps[:, None] * c.T ** 4, c.eps[:, None]], axis=1)
    Y, info = r.rad_solve_reflection(h, c.eps, B, tol=1e-8, refine=True, inner_tol=1e-4)
    assert info["status"] == 0 and info["max_rel_residual"] <= 1e-8
    res = radiosity.residual_rows(f, c.eps, rows, Y, B)
    # residual against the exact operator: the H approximation (ACA 1e-7) dominates
    assert np.linalg.norm(res) / np.linalg.norm(B[rows]) <= 1e-6
    # error bound ||e||_inf <= ||r||_inf / (1 - max(1 - eps) max row sum) on the rows
    s = radiosity.rowsum_rows(f, rows[:64])
    assert s.max() < 1.2
