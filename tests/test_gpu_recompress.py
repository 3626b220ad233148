"""GPU recompression of ACA crosses into standard form with truncated ranks
(§4.3 postprocessing, §5.1 truncation by singular-value decay) against the
oracle's QR + SVD truncation of the very crosses the GPU started from."""
import numpy as np
import pytest

import cavities as cv
from gpu_common import gpu_blocks, rad, rel
from oracle import SIGMA_SB, aca as oaca, geometry, viewfactor

pytestmark = pytest.mark.gpu

# (factor dtype, ACA tol, recompression tol, floating-point noise of a stored
# cross relative to its norm)
CASES = [("f64", 1e-9, 1e-6, 1e-12), ("f32", 1e-6, 1e-4, 3e-6)]


@pytest.fixture(scope="module")
def cyl():
    verts = cv.closed_cylinder(1.0, 4.0, 56, 36, 5)     # 4,592 facets
    return verts, viewfactor.dense(geometry.facets_from_triangles(verts))


def _crosses(h):
    r = rad()
    _, bl, keys = gpu_blocks(h)
    out = {}
    for b, (r0, r1, c0, c1, adm) in enumerate(keys):
        rk = int(bl["rank"][b])
        if adm and rk >= 0:
            out[(r0, r1, c0, c1)] = r.rad_htree_export_block(h, b, r1 - r0, c1 - c0, rk)
    return out


def _oracle_tail(U, V):
    """Singular values of U V^T (oracle QR + SVD) as squared tail sums."""
    _, Ru = np.linalg.qr(U)
    _, Rv = np.linalg.qr(V)
    s = np.linalg.svd(Ru @ Rv.T, compute_uv=False)
    s2 = s * s
    return np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]]), float(s2.sum())


@pytest.mark.parametrize("factor,aca_tol,rc_tol,noise", CASES)
def test_recompression_matches_oracle_truncation(cyl, factor, aca_tol, rc_tol, noise):
    verts, F = cyl
    r = rad()
    h = r.rad_build_htree(verts, 32, 1.0)
    r.rad_compress_aca(h, aca_tol, 64, "partial", factor, factor)
    raw = _crosses(h)
    k_raw = r.rad_htree_get_stats(h)["sum_rank"]
    r.rad_compress_aca(h, aca_tol, 64, "partial", factor, factor, recompress_tol=rc_tol)
    rec = _crosses(h)
    assert raw.keys() == rec.keys()
    n_same = n_cut = n_multi = 0
    for key, (U0, V0) in raw.items():
        U1, V1 = rec[key]
        k0, k1 = U0.shape[1], U1.shape[1]
        X0 = U0 @ V0.T
        nx = np.linalg.norm(X0)
        if k0 < 2:
            assert k1 == k0, key
            np.testing.assert_array_equal(U1 @ V1.T, X0)
            continue
        n_multi += 1
        # truncation error within the requested relative accuracy
        err = np.linalg.norm(U1 @ V1.T - X0)
        assert err <= rc_tol * nx * (1 + 1e-3) + noise * nx, (key, err / nx)
        # the rank is the oracle's smallest admissible rank, up to a value on
        # the threshold within the stored factors' rounding
        Uo, Vo = oaca.truncate(U0, V0, rc_tol)
        ko = Uo.shape[1]
        tail, total = _oracle_tail(U0, V0)
        lim = rc_tol * rc_tol * total
        band = 0.05 * lim + 4 * noise * rc_tol * total
        if k1 != ko:
            assert abs(k1 - ko) == 1, (key, k0, k1, ko)
            assert abs(tail[min(k1, ko)] - lim) <= band, (key, k1, ko, tail[min(k1, ko)] / total, rc_tol ** 2)
        else:
            n_same += 1
            assert rel(U1 @ V1.T, Uo @ Vo.T) <= 2 * rc_tol + 2 * noise, key
        n_cut += k1 < k0
    assert n_multi > 100 and n_same >= 0.98 * n_multi
    assert n_cut > 0
    assert r.rad_htree_get_stats(h)["sum_rank"] < k_raw
    # the recompressed operator still applies F to within ACA + truncation
    x = SIGMA_SB * np.random.default_rng(3).uniform(300.0, 1200.0, size=F.shape[0]) ** 4
    y = r.rad_hmatvec(h, x if factor == "f64" else x.astype(np.float32))
    assert rel(y, F @ x) <= 2 * (aca_tol + rc_tol) + (1e-6 if factor == "f32" else 0.0)


def test_recompression_independent_of_aca_chunking(cyl):
    verts, _ = cyl
    r = rad()
    h = r.rad_build_htree(verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "f32", "f32", recompress_tol=1e-5)
    whole = _crosses(h)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "f32", "f32", scratch_mib=1, recompress_tol=1e-5)
    chunked = _crosses(h)
    assert whole.keys() == chunked.keys()
    for key in whole:
        np.testing.assert_array_equal(whole[key][0], chunked[key][0])
        np.testing.assert_array_equal(whole[key][1], chunked[key][1])


def test_recompression_rejects_bad_tolerance(cyl):
    verts, _ = cyl
    r = rad()
    h = r.rad_build_htree(verts, 32, 1.0)
    for bad in (-1e-3, 1.0, float("nan")):
        with pytest.raises(r.RadError):
            r.rad_compress_aca(h, 1e-6, 64, "partial", "f32", "f32", recompress_tol=bad)
