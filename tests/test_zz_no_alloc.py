"""rad_hmatvec_noalloc, the allocation-free block product.

It exists for callers that cannot let this library allocate device memory
(for example a serving engine that has reserved the GPU's memory for its own
pool).  Here it is called through the C ABI and compared with rad_hmatvec,
the allocating entry point, on several calls in a row (each call reuses the
fixed scratch the one before left behind), with 1, 3, 6 and 65 columns so
that every kernel family of the product runs through the fixed scratch.  This file is collected last on
purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _lib():
    import paper_2305_06891_gb300 as rad
    lib = ctypes.CDLL(rad.LIB_PATH)
    f = lib.rad_hmatvec_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
    return rad, lib


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_matches_allocating_product_on_two_calls(dtype):
    import torch

    import cavities as cv
    rad, lib = _lib()
    verts = cv.closed_cylinder(1.0, 4.0, 40, 24, 4)
    h = rad.rad_build_htree(verts, 24, 1.0)
    rad.rad_compress_aca(h, 1e-7, 64, "partial", dtype, dtype)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    code = rad.RAD_F32 if dtype == "f32" else rad.RAD_F64
    n = h.n
    stream = torch.cuda.current_stream().cuda_stream
    gen = torch.Generator(device="cuda").manual_seed(5)
    # one column, the 2-4 column streaming kernels, and the panel GEMMs of
    # 5 or more columns (6 and 65: padded rows, more than one column chunk)
    for call, nrhs in enumerate((1, 3, 6, 65)):
        X = torch.rand((nrhs, n), device="cuda", dtype=tdt, generator=gen).t()    # column-major
        ref = rad.rad_hmatvec(h, X)
        Y = torch.full((nrhs, n), float("nan"), device="cuda", dtype=tdt).t()
        rc = lib.rad_hmatvec_noalloc(h.ptr.value, code, X.data_ptr(), n, Y.data_ptr(), n, nrhs, stream)
        assert rc == rad.RAD_OK, rad.rad_last_error()
        torch.cuda.synchronize()
        got = Y.cpu().numpy()
        want = ref.cpu().numpy()
        tol = 1e-6 if dtype == "f32" else 1e-12
        for c in range(nrhs):
            err = np.linalg.norm(got[:, c] - want[:, c]) / np.linalg.norm(want[:, c])
            assert err <= tol, (call, c, err)
    rad.rad_htree_free(h)


def test_noalloc_rejects_calls_beyond_its_fixed_scratch():
    import torch

    import cavities as cv
    rad, lib = _lib()
    h = rad.rad_build_htree(cv.unit_cube(8), 32, 1.0)
    rad.rad_compress_aca(h, 1e-6, 64, "partial", "f64", "f64")
    n, nrhs = h.n, 4096
    X = torch.zeros((nrhs, n), device="cuda", dtype=torch.float64).t()
    Y = torch.zeros_like(X)
    rc = lib.rad_hmatvec_noalloc(h.ptr.value, rad.RAD_F64, X.data_ptr(), n, Y.data_ptr(), n, nrhs,
                                 torch.cuda.current_stream().cuda_stream)
    assert rc == rad.RAD_ELIMIT
    assert "fixed scratch" in rad.rad_last_error()
    x = np.zeros(n)
    rc = lib.rad_hmatvec_noalloc(h.ptr.value, rad.RAD_F64, x.ctypes.data, n, Y.data_ptr(), n, 1,
                                 torch.cuda.current_stream().cuda_stream)
    assert rc == rad.RAD_EINVAL
    rad.rad_htree_free(h)
