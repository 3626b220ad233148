"""The flux-solve server: each result is the same alone and in a mix of
overlapping requests (with evictions forced by a small memory budget), and
equals a direct rad_solve_flux call with the same settings."""
import numpy as np
import pytest

import cavities as cv
from gpu_common import rad, rel
from oracle import SIGMA_SB

pytestmark = pytest.mark.gpu

SETTINGS = dict(leaf_size=32, eta_adm=1.0, aca_tol=1e-6, factor_dtype="bf16", near_dtype="f32",
                accurate_dtype="f32", tol=1e-9, refine=True, inner_tol=1e-4)


def _cavities():
    return [cv.unit_cube(8), cv.icosphere(3), cv.box(1.0, 2.0, 3.0, 8, 12, 14), cv.cylinder_for_n(3000)]


def _requests(cavs, count=14):
    rng = cv.rng_for(95)
    out = []
    for k in range(count):
        c = int(rng.integers(0, len(cavs)))
        n = cavs[c].shape[0]
        m = int(rng.integers(1, 3))
        out.append((c, rng.uniform(0.3, 0.9, n), rng.uniform(300.0, 1200.0, (n, m))))
    return out


def _estimate(n):
    # the server's own pre-build estimate for these settings (bytes)
    return n * (900 * 4 + 3500 * 2 + 3500 * 4 + 2048)


def test_alone_equals_mixed_and_direct():
    r = rad()
    cavs = _cavities()
    reqs = _requests(cavs)
    # alone: one slot, one request at a time, budget for everything
    srv = r.Server(slots=1, hbm_budget_bytes=64 << 30, aca_scratch_mib=64, **SETTINGS)
    ids = [srv.add_cavity(v) for v in cavs]
    alone = []
    for c, e, T in reqs:
        q, info = srv.wait(srv.submit(ids[c], e, T))
        assert info["status"] == 0 and info["max_rel_residual"] <= 1e-9
        alone.append(q)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["builds"] == len(set(c for c, _, _ in reqs))
    srv.close()
    # mixed: four slots, everything submitted at once, a budget barely above
    # what building the largest operator reserves (ACA scratch 64 MiB), so
    # that operators are evicted and rebuilt along the way
    big = max(_estimate(v.shape[0]) for v in cavs)
    budget = big + (64 << 20) + (48 << 20)
    srv = r.Server(slots=4, hbm_budget_bytes=budget, aca_scratch_mib=64, **SETTINGS)
    ids = [srv.add_cavity(v) for v in cavs]
    tickets = [srv.submit(ids[c], e, T) for c, e, T in reqs]
    mixed = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["p99_latency_ms"] >= st["p50_latency_ms"] > 0.0
    assert st["evictions"] > 0
    for (q, info), qa in zip(mixed, alone):
        np.testing.assert_array_equal(q, qa)
    # direct call with the same settings
    c, e, T = reqs[0]
    h = r.rad_build_htree(cavs[c], leaf_size=32, eta_adm=1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "bf16", "f32", accurate_dtype="f32", scratch_mib=64)
    qd, _ = r.rad_solve_flux(h, e, T, SIGMA_SB, tol=1e-9, refine=True, inner_tol=1e-4)
    h.free()
    np.testing.assert_array_equal(qd, alone[0])


def test_request_larger_than_budget_fails_cleanly():
    r = rad()
    srv = r.Server(slots=2, hbm_budget_bytes=1 << 20, aca_scratch_mib=64, **SETTINGS)
    cid = srv.add_cavity(cv.unit_cube(4))
    n = cv.unit_cube(4).shape[0]
    t = srv.submit(cid, np.full(n, 0.5), np.full((n, 1), 500.0))
    with pytest.raises(r.RadError):
        srv.wait(t)
    assert srv.stats()["failed"] == 1
    srv.close()


def test_concurrent_builds_with_recompression():
    # four slots build four operators at once, each with recompressed
    # crosses (kernels whose shared-memory size depends on the cavity)
    r = rad()
    cavs = _cavities()
    reqs = [(c, e, T) for c, e, T in _requests(cavs, count=8)]
    srv = r.Server(slots=4, hbm_budget_bytes=64 << 30, aca_scratch_mib=64, recompress_tol=1e-6, **SETTINGS)
    ids = [srv.add_cavity(v) for v in cavs]
    tickets = [srv.submit(ids[c], e, T) for c, e, T in reqs]
    out = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    for q, info in out:
        assert info["status"] == 0 and info["max_rel_residual"] <= 1e-9 and np.isfinite(q).all()
