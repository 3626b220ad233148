"""A batch of cavities in one handle (forest of cluster trees): trees,
blocks, products and solves per cavity equal the single-cavity results, and
the batch flux matches the oracle's direct solve."""
import numpy as np
import pytest

import cavities as cv
from gpu_common import rad, rel
from oracle import SIGMA_SB, geometry, radiosity, viewfactor

pytestmark = pytest.mark.gpu


def _cavities():
    rng = cv.rng_for(90)
    out = []
    for verts in (cv.unit_cube(6), cv.box(1.0, 2.5, 1.5, 5, 9, 6), cv.icosphere(2), cv.unit_cube(1)):
        n = verts.shape[0]
        out.append((verts, rng.uniform(0.3, 0.9, n), rng.uniform(300.0, 1200.0, (n, 2))))
    return out


@pytest.fixture(scope="module")
def batch():
    r = rad()
    cavs = _cavities()
    verts = np.concatenate([c[0] for c in cavs])
    counts = [c[0].shape[0] for c in cavs]
    hb = r.rad_build_htree_batch(verts, counts, leaf_size=16, eta_adm=1.0)
    singles = [r.rad_build_htree(c[0], leaf_size=16, eta_adm=1.0) for c in cavs]
    yield r, cavs, counts, hb, singles
    hb.free()
    for h in singles:
        h.free()


def test_forest_blocks_are_the_single_cavity_blocks(batch):
    r, cavs, counts, hb, singles = batch
    tb, bb = r.rad_htree_export_tree(hb), r.rad_htree_export_blocks(hb)
    off = np.concatenate([[0], np.cumsum(counts)])
    keys_b = set()
    for rn, cn, a in zip(bb["row_node"], bb["col_node"], bb["admissible"]):
        r0, r1, c0, c1 = int(tb["begin"][rn]), int(tb["end"][rn]), int(tb["begin"][cn]), int(tb["end"][cn])
        k = np.searchsorted(off, r0, side="right") - 1
        assert off[k] <= c0 and c1 <= off[k + 1] and r1 <= off[k + 1], "block couples two cavities"
        keys_b.add((r0, r1, c0, c1, bool(a)))
    keys_s = set()
    for k, h in enumerate(singles):
        ts, bs = r.rad_htree_export_tree(h), r.rad_htree_export_blocks(h)
        for rn, cn, a in zip(bs["row_node"], bs["col_node"], bs["admissible"]):
            keys_s.add((int(ts["begin"][rn]) + off[k], int(ts["end"][rn]) + off[k],
                        int(ts["begin"][cn]) + off[k], int(ts["end"][cn]) + off[k], bool(a)))
    assert keys_b == keys_s
    # the tree permutation stays inside each cavity and equals the single one
    perm_b = tb["perm"]
    for k, h in enumerate(singles):
        np.testing.assert_array_equal(perm_b[off[k]:off[k + 1]], r.rad_htree_export_tree(h)["perm"] + off[k])


@pytest.mark.parametrize("fdt", ["f64", "f32"])
def test_batch_product_and_flux_equal_single_cavities(batch, fdt):
    r, cavs, counts, hb, singles = batch
    off = np.concatenate([[0], np.cumsum(counts)])
    tol = 1e-10 if fdt == "f64" else 1e-5
    r.rad_compress_aca(hb, tol, 64, "partial", fdt, fdt)
    for h in singles:
        r.rad_compress_aca(h, tol, 64, "partial", fdt, fdt)
    n = int(off[-1])
    x = np.random.default_rng(3).uniform(0.5, 1.5, (n, 3))
    yb = r.rad_hmatvec(hb, x)
    for k, h in enumerate(singles):
        ys = r.rad_hmatvec(h, x[off[k]:off[k + 1]])
        assert rel(yb[off[k]:off[k + 1]], ys) <= 1e-13
    eps = np.concatenate([c[1] for c in cavs])
    T = np.concatenate([c[2] for c in cavs])
    stol = 1e-10 if fdt == "f64" else 1e-6
    qb, info = r.rad_solve_flux(hb, eps, T, SIGMA_SB, tol=stol)
    assert info["status"] == 0 and info["max_rel_residual"] <= stol
    for k, h in enumerate(singles):
        qs, _ = r.rad_solve_flux(h, cavs[k][1], cavs[k][2], SIGMA_SB, tol=stol)
        assert rel(qb[off[k]:off[k + 1]], qs) <= 1e-12


def test_batch_flux_matches_oracle_direct_solve(batch):
    r, cavs, counts, hb, singles = batch
    off = np.concatenate([[0], np.cumsum(counts)])
    r.rad_compress_aca(hb, 1e-9, 64, "partial", "f64", "f64")
    eps = np.concatenate([c[1] for c in cavs])
    T = np.concatenate([c[2] for c in cavs])
    qb, info = r.rad_solve_flux(hb, eps, T, SIGMA_SB, tol=1e-11)
    for k, (verts, e, Tk) in enumerate(cavs):
        F = viewfactor.dense(geometry.facets_from_triangles(verts))
        q_ref, _, _ = radiosity.solve_flux(F, e, Tk, SIGMA_SB)
        assert rel(qb[off[k]:off[k + 1]], q_ref) <= 1e-6


def test_batch_rejects_bad_counts():
    r = rad()
    v = cv.unit_cube(2)
    with pytest.raises(Exception):
        r.rad_build_htree_batch(v, [v.shape[0], 0])
    with pytest.raises(Exception):
        r.rad_build_htree_batch(v, [v.shape[0] + 1])


def test_chunked_aca_equals_one_pass(batch):
    """A scratch bound of 1 MiB forces the ACA into many chunks (each
    compacted before the next); ranks and products are unchanged."""
    r, cavs, counts, hb, singles = batch
    n = int(sum(counts))
    x = np.random.default_rng(5).uniform(0.5, 1.5, (n, 2))
    r.rad_compress_aca(hb, 1e-6, 64, "partial", "f32", "f32")
    st1, y1 = r.rad_htree_get_stats(hb), r.rad_hmatvec(hb, x)
    r.rad_compress_aca(hb, 1e-6, 64, "partial", "f32", "f32", scratch_mib=1)
    st2, y2 = r.rad_htree_get_stats(hb), r.rad_hmatvec(hb, x)
    for k in ("sum_rank", "far_entries", "near_entries", "aca_entries", "n_dense_fallback"):
        assert st1[k] == st2[k], k
    np.testing.assert_array_equal(y1, y2)


def test_many_cavities_each_converge_like_alone():
    """More virtual columns (cavity x right-hand side) than one CTA of the
    per-column kernels covers: every cavity still solves as it would alone."""
    r = rad()
    rng = cv.rng_for(91)
    cavs = []
    for k in range(90):
        a, b = rng.uniform(1.0, 3.0, 2)
        verts = cv.box(1.0, float(a), float(b), 2, 3, 3)
        n = verts.shape[0]
        cavs.append((verts, rng.uniform(0.3, 0.9, n), rng.uniform(300.0, 1200.0, (n, 1))))
    verts = np.concatenate([c[0] for c in cavs])
    counts = [c[0].shape[0] for c in cavs]
    off = np.concatenate([[0], np.cumsum(counts)])
    hb = r.rad_build_htree_batch(verts, counts, leaf_size=16, eta_adm=1.0)
    r.rad_compress_aca(hb, 1e-10, 64, "partial", "f64", "f64")
    eps = np.concatenate([c[1] for c in cavs])
    T = np.concatenate([c[2] for c in cavs])
    qb, info = r.rad_solve_flux(hb, eps, T, SIGMA_SB, tol=1e-10)
    assert info["status"] == 0 and info["max_rel_residual"] <= 1e-10
    for k in (0, 41, 89):
        h = r.rad_build_htree(cavs[k][0], leaf_size=16, eta_adm=1.0)
        r.rad_compress_aca(h, 1e-10, 64, "partial", "f64", "f64")
        qs, _ = r.rad_solve_flux(h, cavs[k][1], cavs[k][2], SIGMA_SB, tol=1e-10)
        h.free()
        assert rel(qb[off[k]:off[k + 1]], qs) <= 1e-12
    hb.free()
