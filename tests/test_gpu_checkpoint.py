"""Checkpoint and resume of a handle (rad_htree_save / rad_htree_load): the
loaded handle has the same trees, partition and statistics and gives the
same products and solves bit for bit; damaged blobs are rejected."""
import numpy as np
import pytest

import cavities as cv
from gpu_common import rad
from oracle import SIGMA_SB

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", [("f32", "f32", None), ("bf16", "f32", "f32"), ("f64", "f64", None)])
def test_saved_and_loaded_handle_is_identical(storage):
    import torch
    r = rad()
    fac, near, acc = storage
    verts = cv.closed_cylinder(1.0, 4.0, 40, 24, 4)
    rng = np.random.default_rng(2)
    eps = rng.uniform(0.3, 0.9, verts.shape[0])
    T = np.asfortranarray(rng.uniform(300, 1200, (verts.shape[0], 6)))
    h = r.rad_build_htree(verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", fac, near, accurate_dtype=acc)
    r.rad_htree_autotune(h)
    blob = r.rad_htree_save(h)
    x = torch.as_tensor(SIGMA_SB * T ** 4, device="cuda",
                        dtype=torch.float64 if fac == "f64" else torch.float32)
    refine = acc is not None
    ref = [r.rad_hmatvec(h, x).cpu().numpy(), r.rad_hmatvec(h, x[:, 0].contiguous()).cpu().numpy(),
           r.rad_solve_flux(h, eps, T, SIGMA_SB, tol=1e-7, refine=refine)[0]]
    st, tr, bl = r.rad_htree_get_stats(h), r.rad_htree_export_tree(h), r.rad_htree_export_blocks(h)
    h.free()
    g = r.rad_htree_load(blob)
    got = [r.rad_hmatvec(g, x).cpu().numpy(), r.rad_hmatvec(g, x[:, 0].contiguous()).cpu().numpy(),
           r.rad_solve_flux(g, eps, T, SIGMA_SB, tol=1e-7, refine=refine)[0]]
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    assert r.rad_htree_get_stats(g) == st
    for d0, d1 in ((tr, r.rad_htree_export_tree(g)), (bl, r.rad_htree_export_blocks(g))):
        for k in d0:
            assert np.array_equal(d0[k], d1[k]), k
    # saved again: the same blob
    assert r.rad_htree_save(g) == blob
    g.free()


def test_damaged_blobs_are_rejected_and_allocator_is_honoured():
    import torch
    r = rad()
    c = cv.config1()
    h = r.rad_build_htree(c.verts, 32, 1.0)
    r.rad_compress_aca(h, 1e-6, 64, "partial", "f64", "f64")
    blob = r.rad_htree_save(h)
    for bad in (blob[:-1], blob[: len(blob) // 2], blob + b"\0"):
        with pytest.raises(r.RadError) as e:
            r.rad_htree_load(bad)
        assert e.value.code == r.RAD_EINVAL
    al = r.torch_allocator()
    g = r.rad_htree_load(blob, allocator=al)
    assert al.live_bytes > 0
    y0 = r.rad_hmatvec(h, np.ones(c.n))
    y1 = r.rad_hmatvec(g, np.ones(c.n))
    assert np.array_equal(y0, y1)
    g.free()
    torch.cuda.synchronize()
    assert al.live_bytes == 0
    h.free()
