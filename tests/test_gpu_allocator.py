"""Device memory through the caller's allocator (rad_tree_params.allocator),
and host-side fault injection: an allocator that fails, and invalid solve
inputs, each give an error status with nothing leaked and the GPU context
still usable."""
import gc

import numpy as np
import pytest

import cavities as cv
from gpu_common import rad
from oracle import SIGMA_SB

pytestmark = pytest.mark.gpu


def _cavity():
    c = cv.config1()
    T = np.asfortranarray(c.T[:, :1] * np.array([1.0, 0.9, 1.1]))   # three fields
    return c.verts, c.eps, T


def _run(r, verts, eps, T, allocator=None):
    import torch
    h = r.rad_build_htree(torch.as_tensor(verts, device="cuda"), 32, 1.0, allocator=allocator)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "f32", "f32")
    x = torch.as_tensor(SIGMA_SB * T ** 4, device="cuda", dtype=torch.float32)
    y = r.rad_hmatvec(h, x).cpu().numpy()
    q, info = r.rad_solve_flux(h, torch.as_tensor(eps, device="cuda"), torch.as_tensor(T, device="cuda"),
                               SIGMA_SB, tol=1e-6)
    assert info["status"] == 0
    return h, y, q.cpu().numpy()


def test_every_handle_buffer_comes_from_torch_caching_allocator():
    import torch
    r = rad()
    verts, eps, T = _cavity()
    _, y0, q0 = _run(r, verts, eps, T)
    gc.collect()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    al = r.torch_allocator()
    h, y1, q1 = _run(r, verts, eps, T, allocator=al)
    torch.cuda.synchronize()
    st = r.rad_htree_get_stats(h)
    # the handle holds its operator (and index lists) in torch's pool
    assert al.live_bytes >= st["bytes_near"] + st["bytes_far"]
    assert torch.cuda.memory_allocated() - base >= al.live_bytes
    # per-call workspaces came from the callback too and went back
    assert al.n_alloc > len(al.live)
    # same kernels on the same bits: identical results
    assert np.array_equal(y0, y1) and np.array_equal(q0, q1)
    r.rad_htree_free(h)
    gc.collect()
    torch.cuda.synchronize()
    assert al.live_bytes == 0 and not al.live and al.n_alloc == al.n_free
    assert torch.cuda.memory_allocated() == base


@pytest.mark.parametrize("fail_after", [0, 2, 9, 40])
def test_failing_allocator_gives_enomem_and_leaks_nothing(fail_after):
    import torch
    r = rad()
    verts, eps, T = _cavity()
    al = r.torch_allocator(fail_after=fail_after)
    vd = torch.as_tensor(verts, device="cuda")
    gc.collect()          # tensors other tests left to the collector
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    h = None
    with pytest.raises(r.RadError) as e:
        h = r.rad_build_htree(vd, 32, 1.0, allocator=al)
        r.rad_compress_aca(h, 1e-6, 64, "partial", "f32", "f32")
        r.rad_solve_flux(h, eps, T, SIGMA_SB, tol=1e-6)
    assert e.value.code == r.RAD_ENOMEM
    assert "allocator" in r.rad_last_error()
    if h is not None:
        r.rad_htree_free(h)
    del e
    gc.collect()
    torch.cuda.synchronize()
    assert al.live_bytes == 0 and al.n_alloc == al.n_free
    assert torch.cuda.memory_allocated() == base
    # the context is fine: a fresh handle on the library's pool works
    _, y, q = _run(r, verts, eps, T)
    assert np.isfinite(q).all()


def test_invalid_solve_inputs_are_rejected_before_solving():
    import torch
    r = rad()
    verts, eps, T = _cavity()
    h, _, q_ok = _run(r, verts, eps, T)
    l0 = r.rad_launch_count()
    for bad_eps, bad_T in [(np.nan, None), (0.0, None), (1.5, None), (None, np.inf), (None, -1.0)]:
        e2, T2 = eps.copy(), T.copy()
        if bad_eps is not None:
            e2[17] = bad_eps
        if bad_T is not None:
            T2[5, 1] = bad_T
        for dev in (False, True):
            ea = torch.as_tensor(e2, device="cuda") if dev else e2
            Ta = torch.as_tensor(np.asfortranarray(T2), device="cuda") if dev else T2
            with pytest.raises(r.RadError) as ex:
                r.rad_solve_flux(h, ea, Ta, SIGMA_SB, tol=1e-6)
            assert ex.value.code == r.RAD_EINVAL
    # only the input checks ran (one launch each), no solver kernel
    assert r.rad_launch_count() - l0 == 10
    B = np.ones((h.n, 2))
    B[3, 1] = np.nan
    with pytest.raises(r.RadError) as ex:
        r.rad_solve_reflection(h, eps, B, tol=1e-8)
    assert ex.value.code == r.RAD_EINVAL
    # the handle still solves correctly afterwards
    q, info = r.rad_solve_flux(h, eps, T, SIGMA_SB, tol=1e-6)
    assert info["status"] == 0 and np.array_equal(q, q_ok)
    r.rad_htree_free(h)


def test_server_takes_every_operator_and_workspace_from_the_allocator():
    import torch
    r = rad()
    verts, eps, T = _cavity()
    results = []
    for al in (None, r.torch_allocator()):
        srv = r.Server(slots=2, hbm_budget_bytes=8 << 30, leaf_size=32, aca_tol=1e-6, factor_dtype="f32",
                       near_dtype="f32", accurate_dtype=None, tol=1e-6, refine=False, aca_scratch_mib=256,
                       allocator=al)
        cid = srv.add_cavity(verts)
        tickets = [srv.submit(cid, eps, T[:, k:k + 1], SIGMA_SB) for k in range(3)]
        results.append([srv.wait(t)[0] for t in tickets])
        if al is not None:
            assert al.n_alloc > 0 and al.live_bytes > 0     # the resident operator
        srv.close()
        torch.cuda.synchronize()
        if al is not None:
            assert al.live_bytes == 0 and al.n_alloc == al.n_free
    for a, b in zip(*results):
        assert np.array_equal(a, b)
