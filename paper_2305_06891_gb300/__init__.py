"""GB300 hierarchical block low-rank cavity radiation.

Thin Python binding of the C ABI in ``include/rad.h`` (``librad.so``).  The
functions carry the C names and only marshal arguments: every step of the
hot path (geometry, trees, ACA, block matrix products, GMRES, flux) runs in
the library's CUDA kernels.  There is no CPU fallback: importing this module
fails loudly (ImportError at the first call) when the compiled library is
missing; build it with ``python -m paper_2305_06891_gb300.build``.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); matrices
are passed column-major (the binding makes a column-major copy when needed).
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# RAD_LIB=checked loads the bounds-checked build (librad_checked.so: canary
# words around every device allocation, verified after every call)
LIB_PATH = os.path.join(_HERE, "librad_checked.so" if os.environ.get("RAD_LIB") == "checked" else "librad.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "rad.h")

SIGMA_SB = 5.670374419e-8

RAD_OK, RAD_EINVAL, RAD_ENOMEM, RAD_ENOTCONV, RAD_ECUDA, RAD_ELIMIT = range(6)
RAD_F64, RAD_F32, RAD_BF16 = 0, 1, 2
RAD_ACA_PARTIAL, RAD_ACA_FULL = 0, 1
_DT = {"f64": RAD_F64, "f32": RAD_F32, "bf16": RAD_BF16}
_PIV = {"partial": RAD_ACA_PARTIAL, "full": RAD_ACA_FULL}


class RadError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"librad error {code}: {msg}")
        self.code = code


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p)


class _Allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", C.c_void_p)]


class _TreeParams(C.Structure):
    _fields_ = [("leaf_size", C.c_int32), ("reserved", C.c_int32), ("eta_adm", C.c_double),
                ("allocator", C.POINTER(_Allocator))]


class Allocator:
    """Device memory of a handle through the caller's callbacks
    (``rad_allocator``): ``alloc(nbytes, stream) -> int`` returns a device
    pointer (0 or an exception: allocation failure, the library call returns
    RAD_ENOMEM) and ``free(ptr, nbytes, stream)`` takes it back; ``stream`` is
    the cudaStream_t of the library call as an int.  Counts what is live.
    ``fail_after`` makes every allocation after the first ``fail_after`` fail
    (fault injection for tests)."""

    def __init__(self, alloc, free, fail_after: int | None = None):
        self.n_alloc = self.n_free = 0
        self.live_bytes = self.peak_bytes = 0
        self.live: dict[int, int] = {}
        self.fail_after = fail_after

        def _a(ctx, nbytes, stream):
            try:
                if self.fail_after is not None and self.n_alloc >= self.fail_after:
                    return None
                ptr = int(alloc(int(nbytes), int(stream or 0)))
            except Exception:
                return None
            if ptr:
                self.n_alloc += 1
                self.live[ptr] = int(nbytes)
                self.live_bytes += int(nbytes)
                self.peak_bytes = max(self.peak_bytes, self.live_bytes)
            return ptr or None

        def _f(ctx, ptr, nbytes, stream):
            try:
                self.n_free += 1
                self.live_bytes -= self.live.pop(int(ptr), 0)
                free(int(ptr), int(nbytes), int(stream or 0))
            except Exception:
                pass

        self._cb = (_ALLOC_FN(_a), _FREE_FN(_f))
        self.struct = _Allocator(self._cb[0], self._cb[1], None)


def torch_allocator(device=None, fail_after: int | None = None) -> Allocator:
    """The PyTorch caching allocator as a handle's device memory: every
    buffer of the handle and every workspace of calls on it is a block of
    torch's pool (``torch.cuda.memory_allocated`` counts it), allocated for
    the library call's stream."""
    t = _torch()
    dev = t.cuda.current_device() if device is None else t.device(device).index

    def alloc(nbytes, stream):
        return t.cuda.caching_allocator_alloc(nbytes, device=dev, stream=stream)

    def free(ptr, nbytes, stream):
        t.cuda.caching_allocator_delete(ptr)

    return Allocator(alloc, free, fail_after)


def _tree_params(leaf_size, eta_adm, allocator):
    p = _TreeParams(int(leaf_size), 0, float(eta_adm), None)
    if allocator is not None:
        p.allocator = C.pointer(allocator.struct)
    return p


class _AcaParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_rank", C.c_int32), ("pivoting", C.c_int32),
                ("factor_dtype", C.c_int32), ("near_dtype", C.c_int32), ("accurate_dtype", C.c_int32),
                ("scratch_mib", C.c_int32), ("recompress_tol", C.c_double)]


class _SolveParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int32), ("max_iter", C.c_int32), ("refine", C.c_int32),
                ("max_refine", C.c_int32), ("inner_tol", C.c_double), ("precond", C.c_void_p)]


class _HluParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("reserved0", C.c_int32), ("reserved1", C.c_int32)]


class _HluStats(C.Structure):
    _fields_ = [("n", C.c_int64), ("dense_entries", C.c_int64), ("lowrank_entries", C.c_int64),
                ("max_rank", C.c_int32), ("n_lowrank", C.c_int32), ("n_dense_fallback", C.c_int32),
                ("precision", C.c_int32), ("tol", C.c_double), ("factor_ms", C.c_double),
                ("solve_launches", C.c_int32), ("reserved", C.c_int32)]


class _SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("restarts", C.c_int32),
                ("matvecs", C.c_int32), ("max_rel_residual", C.c_double), ("refinements", C.c_int32),
                ("reserved", C.c_int32)]


class _ServerParams(C.Structure):
    _fields_ = [("slots", C.c_int32), ("reserved", C.c_int32), ("hbm_budget_bytes", C.c_int64),
                ("tree", _TreeParams), ("aca", _AcaParams), ("solve", _SolveParams)]


class _RequestInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("built", C.c_int32), ("iters", C.c_int32), ("refinements", C.c_int32),
                ("max_rel_residual", C.c_double), ("queue_ms", C.c_double), ("service_ms", C.c_double),
                ("latency_ms", C.c_double), ("slot", C.c_int32), ("reserved", C.c_int32)]


class _ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("builds", C.c_int64), ("evictions", C.c_int64), ("resident_bytes", C.c_int64),
                ("peak_bytes", C.c_int64), ("resident_cavities", C.c_int32), ("in_flight", C.c_int32),
                ("p50_latency_ms", C.c_double), ("p99_latency_ms", C.c_double), ("max_latency_ms", C.c_double),
                ("mean_service_ms", C.c_double)]


class _Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("leaf_size", C.c_int32), ("n_nodes", C.c_int32),
                ("n_leaf_clusters", C.c_int32), ("depth", C.c_int32), ("n_blocks", C.c_int64),
                ("n_admissible", C.c_int64), ("compressed", C.c_int32), ("factor_dtype", C.c_int32),
                ("near_dtype", C.c_int32), ("max_rank_used", C.c_int32), ("n_dense_fallback", C.c_int64),
                ("near_entries", C.c_int64), ("far_entries", C.c_int64), ("sum_rank", C.c_int64),
                ("aca_entries", C.c_int64), ("bytes_near", C.c_int64), ("bytes_far", C.c_int64),
                ("far_u_entries", C.c_int64), ("far_v_entries", C.c_int64), ("n_tiles", C.c_int64),
                ("bytes_accurate", C.c_int64), ("tuned", C.c_int32), ("stream_rows", C.c_int32),
                ("grid_a1", C.c_int32), ("grid_b1", C.c_int32), ("grid_a2", C.c_int32), ("grid_b2", C.c_int32),
                ("product_path", C.c_int32), ("closed", C.c_int32), ("one_column_path", C.c_int32),
                ("reserved", C.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2305_06891_gb300.build` "
                          "(this package has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    H = C.c_void_p
    sig = {
        "rad_version": (C.c_int, []),
        "rad_debug_bounds_checks": (C.c_int, []),
        "rad_last_error": (C.c_char_p, []),
        "rad_build_htree": (C.c_int, [i64, vp, C.POINTER(_TreeParams), vp, C.POINTER(H)]),
        "rad_build_htree_facets": (C.c_int, [i64, vp, vp, vp, C.POINTER(_TreeParams), vp, C.POINTER(H)]),
        "rad_build_htree_batch": (C.c_int, [i32, vp, vp, C.POINTER(_TreeParams), vp, C.POINTER(H)]),
        "rad_htree_from_dense": (C.c_int, [i64, vp, vp, C.POINTER(H)]),
        "rad_compress_aca": (C.c_int, [H, C.POINTER(_AcaParams), vp]),
        "rad_hmatvec": (C.c_int, [H, i32, vp, i64, vp, i64, i64, vp]),
        "rad_solve_flux": (C.c_int, [H, vp, vp, i64, i64, dbl, C.POINTER(_SolveParams), vp, i64,
                                     C.POINTER(_SolveInfo), vp]),
        "rad_hmatvec_noalloc": (C.c_int, [H, i32, vp, i64, vp, i64, i64, vp]),
        "rad_solve_reflection": (C.c_int, [H, vp, vp, i64, i64, C.POINTER(_SolveParams), vp, i64,
                                           C.POINTER(_SolveInfo), vp]),
        "rad_htree_get_stats": (C.c_int, [H, C.POINTER(_Stats)]),
        "rad_htree_export_tree": (C.c_int, [H, vp, vp, vp, vp, vp, vp]),
        "rad_htree_export_blocks": (C.c_int, [H, vp, vp, vp, vp]),
        "rad_htree_export_block": (C.c_int, [H, i64, vp, vp, vp]),
        "rad_htree_free": (C.c_int, [H]),
        "rad_htree_autotune": (C.c_int, [H, vp]),
        "rad_htree_set_product_path": (C.c_int, [H, i32]),
        "rad_htree_set_one_column_path": (C.c_int, [H, i32]),
        "rad_htree_close_cavity": (C.c_int, [H, vp, vp]),
        "rad_server_create": (C.c_int, [C.POINTER(_ServerParams), C.POINTER(vp)]),
        "rad_server_add_cavity": (C.c_int, [vp, i64, vp, C.POINTER(i64)]),
        "rad_server_submit": (C.c_int, [vp, i64, vp, vp, i64, i64, dbl, vp, i64, C.POINTER(i64)]),
        "rad_server_wait": (C.c_int, [vp, i64, C.POINTER(_RequestInfo)]),
        "rad_server_get_stats": (C.c_int, [vp, C.POINTER(_ServerStats)]),
        "rad_server_destroy": (C.c_int, [vp]),
        "rad_htree_save": (C.c_int, [H, vp, C.POINTER(C.c_uint64)]),
        "rad_htree_load": (C.c_int, [vp, C.c_uint64, C.POINTER(_TreeParams), vp, C.POINTER(H)]),
        "rad_hlu_factor": (C.c_int, [H, vp, C.POINTER(_HluParams), vp, C.POINTER(vp)]),
        "rad_hlu_solve": (C.c_int, [vp, vp, i64, i64, vp, i64, vp]),
        "rad_hlu_get_stats": (C.c_int, [vp, C.POINTER(_HluStats)]),
        "rad_hlu_export": (C.c_int, [vp, vp]),
        "rad_hlu_free": (C.c_int, [vp]),
        "rad_launch_count": (C.c_int64, []),
        "rad_profile_enable": (C.c_int, [i32]),
        "rad_profile_read": (C.c_int, [i32, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


class _LazyLib:
    """Loads librad.so on first use; raises ImportError if it is missing."""
    _h = None

    def __getattr__(self, name):
        if _LazyLib._h is None:
            _LazyLib._h = _load()
        return getattr(_LazyLib._h, name)


_lib = _LazyLib()


def load_library():
    """Load librad.so now (raises ImportError when it has not been built)."""
    _lib.rad_version()
    return LIB_PATH


def header_functions() -> list[str]:
    """Names of every function declared in include/rad.h."""
    txt = open(HEADER_PATH).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*|void)\s+(rad_\w+)\s*\(", txt, re.M)))


def _check(rc: int):
    if rc != RAD_OK:
        raise RadError(rc, _lib.rad_last_error().decode())


def _torch():
    try:
        import torch
        return torch
    except ImportError:  # pragma: no cover
        return None


def _is_tensor(a) -> bool:
    t = _torch()
    return t is not None and isinstance(a, t.Tensor)


def _stream(stream, *arrays):
    if stream is not None:
        return C.c_void_p(int(stream))
    t = _torch()
    if t is not None and any(_is_tensor(a) and a.is_cuda for a in arrays):
        return C.c_void_p(t.cuda.current_stream().cuda_stream)
    return C.c_void_p(0)


def _ptr(a) -> C.c_void_p:
    if _is_tensor(a):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def _f64_rowmajor(a, shape_last: int | None = None):
    """float64, C-contiguous (tensor or numpy)."""
    if _is_tensor(a):
        t = _torch()
        return a.to(t.float64).contiguous()
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _colmajor(a, dtype):
    """2-D column-major copy/view with the requested element type; returns
    (array, n_rows, n_cols, ld)."""
    if _is_tensor(a):
        t = _torch()
        td = {np.float64: t.float64, np.float32: t.float32}[dtype]
        a2 = a.reshape(-1, 1) if a.dim() == 1 else a
        a2 = a2.to(td)
        if a2.stride(0) != 1 or (a2.shape[1] > 1 and a2.stride(1) < a2.shape[0]):
            a2 = a2.t().contiguous().t()
        ld = a2.stride(1) if a2.shape[1] > 1 else a2.shape[0]
        return a2, a2.shape[0], a2.shape[1], max(ld, a2.shape[0])
    a2 = np.asarray(a, dtype=dtype)
    if a2.ndim == 1:
        a2 = a2.reshape(-1, 1)
    a2 = np.asfortranarray(a2)
    return a2, a2.shape[0], a2.shape[1], a2.shape[0]


class HTree:
    """Owns one ``rad_htree*``; freed with :func:`rad_htree_free` or on GC.
    Keeps the handle's :class:`Allocator` (if any) alive with it."""

    def __init__(self, ptr: int, n: int, allocator: Allocator | None = None):
        self._p = C.c_void_p(ptr)
        self.n = n
        self.allocator = allocator

    @property
    def ptr(self) -> C.c_void_p:
        if not self._p:
            raise RadError(RAD_EINVAL, "handle already freed")
        return self._p

    def free(self):
        if self._p:
            _lib.rad_htree_free(self._p)
            self._p = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def rad_version() -> int:
    return _lib.rad_version()


def rad_debug_bounds_checks() -> bool:
    """True when the loaded library is the bounds-checked build."""
    return bool(_lib.rad_debug_bounds_checks())


def rad_last_error() -> str:
    return _lib.rad_last_error().decode()


def rad_build_htree(verts, leaf_size: int = 32, eta_adm: float = 1.0, stream=None,
                    allocator: Allocator | None = None) -> HTree:
    """A1-A3 on the GPU: facets of the triangles ``verts`` (N, 3, 3).
    ``allocator``: device memory of the handle (default: the library's pool)."""
    v = _f64_rowmajor(verts)
    n = int(v.shape[0])
    out = C.c_void_p()
    p = _tree_params(leaf_size, eta_adm, allocator)
    _check(_lib.rad_build_htree(n, _ptr(v), C.byref(p), _stream(stream, v), C.byref(out)))
    return HTree(out.value, n, allocator)


def rad_build_htree_batch(verts, counts, leaf_size: int = 32, eta_adm: float = 1.0, stream=None,
                          allocator: Allocator | None = None) -> HTree:
    """A batch of cavities in one handle: ``verts`` (sum(counts), 3, 3) holds the
    cavities' triangles one cavity after the other, ``counts`` their numbers."""
    v = _f64_rowmajor(verts)
    cnt = np.ascontiguousarray(np.asarray(counts, dtype=np.int64))
    n = int(v.shape[0])
    if int(cnt.sum()) != n:
        raise ValueError("sum(counts) must equal the number of triangles")
    out = C.c_void_p()
    p = _tree_params(leaf_size, eta_adm, allocator)
    _check(_lib.rad_build_htree_batch(int(cnt.size), cnt.ctypes.data, _ptr(v), C.byref(p), _stream(stream, v),
                                      C.byref(out)))
    return HTree(out.value, n, allocator)


def rad_build_htree_facets(centroid, normal, area, leaf_size: int = 32, eta_adm: float = 1.0,
                           stream=None, allocator: Allocator | None = None) -> HTree:
    c, nr, a = _f64_rowmajor(centroid), _f64_rowmajor(normal), _f64_rowmajor(area)
    n = int(a.shape[0])
    out = C.c_void_p()
    p = _tree_params(leaf_size, eta_adm, allocator)
    _check(_lib.rad_build_htree_facets(n, _ptr(c), _ptr(nr), _ptr(a), C.byref(p), _stream(stream, c),
                                       C.byref(out)))
    return HTree(out.value, n, allocator)


def rad_htree_from_dense(F, stream=None) -> HTree:
    Fm = _f64_rowmajor(F)
    n = int(Fm.shape[0])
    out = C.c_void_p()
    _check(_lib.rad_htree_from_dense(n, _ptr(Fm), _stream(stream, Fm), C.byref(out)))
    return HTree(out.value, n)


def rad_compress_aca(h: HTree, tol: float, max_rank: int = 64, pivoting: str = "partial",
                     factor_dtype: str = "f32", near_dtype: str = "f32", accurate_dtype: str | None = None,
                     stream=None, scratch_mib: int = 0, recompress_tol: float = 0.0) -> None:
    """ACA of the admissible blocks (dense entries for the others).
    ``recompress_tol`` > 0 truncates every cross to standard form at that
    relative accuracy (SVD of R_U R_V^T after QR of both factors)."""
    acc = -1 if accurate_dtype is None else _DT[accurate_dtype]
    p = _AcaParams(float(tol), int(max_rank), _PIV[pivoting], _DT[factor_dtype], _DT[near_dtype], acc,
                   int(scratch_mib), float(recompress_tol))
    _check(_lib.rad_compress_aca(h.ptr, C.byref(p), _stream(stream)))


def rad_hmatvec(h: HTree, x, y=None, stream=None):
    """Y = F X.  ``x``: (N,) or (N, nrhs), float64 or float32, host or device."""
    is_t = _is_tensor(x)
    if is_t:
        t = _torch()
        dt = np.float64 if x.dtype == t.float64 else np.float32
    else:
        dt = np.float64 if np.asarray(x).dtype == np.float64 else np.float32
    xc, n, nrhs, ldx = _colmajor(x, dt)
    y_given = y is not None
    if y is None:
        if is_t:
            y = t.empty((nrhs, n), dtype=xc.dtype, device=xc.device).t()
        else:
            y = np.empty((n, nrhs), dtype=dt, order="F")
        ldy = n
    else:
        ldy = (y.stride(1) if y.dim() == 2 else n) if _is_tensor(y) else n
    _check(_lib.rad_hmatvec(h.ptr, RAD_F64 if dt == np.float64 else RAD_F32, _ptr(xc), ldx, _ptr(y), ldy,
                            nrhs, _stream(stream, xc, y)))
    one_d = (_is_tensor(x) and x.dim() == 1) or (not _is_tensor(x) and np.ndim(x) == 1)
    if one_d and not y_given:
        return y[:, 0]
    return y


def rad_solve_flux(h: HTree, eps, T, sigma: float = SIGMA_SB, tol: float = 1e-10, restart: int = 30,
                   max_iter: int = 1000, q=None, stream=None, raise_on_notconv: bool = False,
                   refine: bool = False, inner_tol: float = 1e-4, max_refine: int = 10, precond=None):
    """A7-A8: flux q (N, m) for temperature fields T (N,) or (N, m).

    Returns ``(q, info)``; ``info`` is a dict with status, iters, restarts,
    matvecs and max_rel_residual.
    """
    Tc, n, m, ldT = _colmajor(T, np.float64)
    e = _f64_rowmajor(eps)
    if q is None:
        if _is_tensor(Tc):
            t = _torch()
            q = t.empty((m, n), dtype=t.float64, device=Tc.device).t()
        else:
            q = np.empty((n, m), dtype=np.float64, order="F")
    ldq = n
    p = _SolveParams(float(tol), int(restart), int(max_iter), 1 if refine else 0, int(max_refine), float(inner_tol),
                     precond.ptr if precond is not None else None)
    info = _SolveInfo()
    rc = _lib.rad_solve_flux(h.ptr, _ptr(e), _ptr(Tc), ldT, m, float(sigma), C.byref(p), _ptr(q), ldq,
                             C.byref(info), _stream(stream, e, Tc, q))
    if rc != RAD_OK and (rc != RAD_ENOTCONV or raise_on_notconv):
        _check(rc)
    d = {k: getattr(info, k) for k, _ in _SolveInfo._fields_}
    if (_is_tensor(T) and T.dim() == 1) or (not _is_tensor(T) and np.ndim(T) == 1):
        q = q[:, 0]
    return q, d


def rad_hmatvec_noalloc(h: HTree, x, y, stream=None):
    """Y = F X without device allocation (fixed 32 MiB scratch per GPU).

    For callers that cannot let the library allocate device memory.  ``x``
    and ``y`` must be CUDA tensors, (N,) or (N, nrhs) column-major, of the
    same dtype (float32 or float64); ``y`` is written in place.
    """
    t = _torch()
    dt = RAD_F64 if x.dtype == t.float64 else RAD_F32
    n = x.shape[0]
    nrhs = 1 if x.dim() == 1 else x.shape[1]
    ldx = n if x.dim() == 1 or nrhs == 1 else x.stride(1)
    ldy = n if y.dim() == 1 or nrhs == 1 else y.stride(1)
    _check(_lib.rad_hmatvec_noalloc(h.ptr, dt, _ptr(x), ldx, _ptr(y), ldy, nrhs, _stream(stream, x, y)))
    return y


def rad_solve_reflection(h: HTree, eps, B, tol: float = 1e-10, restart: int = 30, max_iter: int = 1000,
                         Y=None, stream=None, raise_on_notconv: bool = False, refine: bool = False,
                         inner_tol: float = 1e-4, max_refine: int = 10, precond=None):
    """A7: Y solving C Y = B (Eq. 11) for B (N,) or (N, nrhs).  Returns (Y, info)."""
    Bc, n, nrhs, ldB = _colmajor(B, np.float64)
    e = _f64_rowmajor(eps)
    if Y is None:
        if _is_tensor(Bc):
            t = _torch()
            Y = t.empty((nrhs, n), dtype=t.float64, device=Bc.device).t()
        else:
            Y = np.empty((n, nrhs), dtype=np.float64, order="F")
    p = _SolveParams(float(tol), int(restart), int(max_iter), 1 if refine else 0, int(max_refine), float(inner_tol),
                     precond.ptr if precond is not None else None)
    info = _SolveInfo()
    rc = _lib.rad_solve_reflection(h.ptr, _ptr(e), _ptr(Bc), ldB, nrhs, C.byref(p), _ptr(Y), n, C.byref(info),
                                   _stream(stream, e, Bc, Y))
    if rc != RAD_OK and (rc != RAD_ENOTCONV or raise_on_notconv):
        _check(rc)
    d = {k: getattr(info, k) for k, _ in _SolveInfo._fields_}
    if (_is_tensor(B) and B.dim() == 1) or (not _is_tensor(B) and np.ndim(B) == 1):
        Y = Y[:, 0]
    return Y, d


class HLU:
    """Owns one ``rad_hlu*`` (block LU factors of the reflection matrix);
    keeps its handle alive, freed with :func:`rad_hlu_free` or on GC."""

    def __init__(self, ptr: int, h: HTree):
        self._p = C.c_void_p(ptr)
        self.h = h
        self.n = h.n

    @property
    def ptr(self) -> C.c_void_p:
        if not self._p:
            raise RadError(RAD_EINVAL, "factors already freed")
        return self._p

    def free(self):
        if self._p:
            _lib.rad_hlu_free(self._p)
            self._p = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def rad_hlu_factor(h: HTree, eps, tol: float, stream=None) -> HLU:
    """§5.1: block LU of C = I - diag(1 - eps) F (the handle's stored F) with
    the ranks of the admissible leaves truncated at ``tol``."""
    e = _f64_rowmajor(eps)
    p = _HluParams(float(tol), 0, 0)
    out = C.c_void_p()
    _check(_lib.rad_hlu_factor(h.ptr, _ptr(e), C.byref(p), _stream(stream, e), C.byref(out)))
    return HLU(out.value, h)


def rad_hlu_solve(lu: HLU, B, X=None, stream=None):
    """§5.2: X = U^-1 L^-1 B by forward and backward substitution through the
    block structure.  ``B`` (N,) or (N, nrhs), host or device."""
    Bc, n, nrhs, ldB = _colmajor(B, np.float64)
    if X is None:
        if _is_tensor(Bc):
            t = _torch()
            X = t.empty((nrhs, n), dtype=t.float64, device=Bc.device).t()
        else:
            X = np.empty((n, nrhs), dtype=np.float64, order="F")
    _check(_lib.rad_hlu_solve(lu.ptr, _ptr(Bc), ldB, nrhs, _ptr(X), n, _stream(stream, Bc, X)))
    if (_is_tensor(B) and B.dim() == 1) or (not _is_tensor(B) and np.ndim(B) == 1):
        X = X[:, 0]
    return X


def rad_hlu_get_stats(lu: HLU) -> dict:
    st = _HluStats()
    _check(_lib.rad_hlu_get_stats(lu.ptr, C.byref(st)))
    return {k: getattr(st, k) for k, _ in _HluStats._fields_}


def rad_hlu_export(lu: HLU) -> np.ndarray:
    """The factors as one dense (N, N) array in tree order: L strictly below
    the diagonal (unit diagonal), U on and above it."""
    out = np.empty((lu.n, lu.n), dtype=np.float64)
    _check(_lib.rad_hlu_export(lu.ptr, out.ctypes.data))
    return out


def rad_hlu_free(lu: HLU) -> None:
    lu.free()


class Server:
    """Flux-solve server (continuous batching over resident operators; see
    ``rad_server_create``).  Host arrays only; ``submit`` keeps references to
    its arrays until ``wait`` returns the flux."""

    def __init__(self, slots: int = 4, hbm_budget_bytes: int = 64 << 30, leaf_size: int = 64,
                 eta_adm: float = 1.0, aca_tol: float = 1e-6, max_rank: int = 64, factor_dtype: str = "bf16",
                 near_dtype: str = "f32", accurate_dtype: str | None = "f32", tol: float = 1e-8,
                 restart: int = 30, max_iter: int = 1000, refine: bool = True, inner_tol: float = 1e-4,
                 max_refine: int = 10, aca_scratch_mib: int = 0, recompress_tol: float = 0.0,
                 allocator: Allocator | None = None):
        acc = -1 if accurate_dtype is None else _DT[accurate_dtype]
        self.allocator = allocator
        p = _ServerParams(int(slots), 0, int(hbm_budget_bytes), _tree_params(leaf_size, eta_adm, allocator),
                          _AcaParams(float(aca_tol), int(max_rank), RAD_ACA_PARTIAL, _DT[factor_dtype],
                                     _DT[near_dtype], acc, int(aca_scratch_mib), float(recompress_tol)),
                          _SolveParams(float(tol), int(restart), int(max_iter), 1 if refine else 0,
                                       int(max_refine), float(inner_tol)))
        out = C.c_void_p()
        _check(_lib.rad_server_create(C.byref(p), C.byref(out)))
        self._p = out
        self._keep = {}
        self._n = []

    def add_cavity(self, verts) -> int:
        v = _f64_rowmajor(verts)
        cid = C.c_int64()
        _check(_lib.rad_server_add_cavity(self._p, int(v.shape[0]), _ptr(v), C.byref(cid)))
        self._n.append(int(v.shape[0]))
        return int(cid.value)

    def submit(self, cavity_id: int, eps, T, sigma: float = SIGMA_SB) -> int:
        n = self._n[cavity_id]
        e = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
        Tm = np.asfortranarray(np.asarray(T, dtype=np.float64).reshape(n, -1))
        q = np.empty(Tm.shape, dtype=np.float64, order="F")
        t = C.c_int64()
        _check(_lib.rad_server_submit(self._p, int(cavity_id), _ptr(e), _ptr(Tm), n, int(Tm.shape[1]),
                                      float(sigma), _ptr(q), n, C.byref(t)))
        self._keep[int(t.value)] = (e, Tm, q)
        return int(t.value)

    def wait(self, ticket: int):
        info = _RequestInfo()
        rc = _lib.rad_server_wait(self._p, int(ticket), C.byref(info))
        e, Tm, q = self._keep.pop(int(ticket))
        d = {k: getattr(info, k) for k, _ in _RequestInfo._fields_}
        if rc not in (RAD_OK, RAD_ENOTCONV):
            raise RadError(rc, f"request {ticket} failed: status {rc}")
        return q, d

    def stats(self) -> dict:
        st = _ServerStats()
        _check(_lib.rad_server_get_stats(self._p, C.byref(st)))
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_}

    def close(self):
        if self._p:
            _lib.rad_server_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rad_server_create(**kw) -> Server:
    """Same-name wrapper of the C entry point: a new :class:`Server`."""
    return Server(**kw)


def rad_server_add_cavity(server: Server, verts) -> int:
    return server.add_cavity(verts)


def rad_server_submit(server: Server, cavity_id: int, eps, T, sigma: float = SIGMA_SB) -> int:
    return server.submit(cavity_id, eps, T, sigma)


def rad_server_wait(server: Server, ticket: int):
    return server.wait(ticket)


def rad_server_get_stats(server: Server) -> dict:
    return server.stats()


def rad_server_destroy(server: Server) -> None:
    server.close()


def rad_htree_autotune(h: HTree, stream=None) -> dict:
    """Choose the streaming products' item rows and grids by timing them on
    this handle's operator; returns the chosen configuration."""
    _check(_lib.rad_htree_autotune(h.ptr, _stream(stream)))
    st = rad_htree_get_stats(h)
    return {k: st[k] for k in ("stream_rows", "grid_a1", "grid_b1", "grid_a2", "grid_b2", "product_path",
                               "one_column_path")}


def rad_htree_close_cavity(h: HTree, stream=None) -> np.ndarray:
    """Closed-cavity row normalisation (§6); returns the row sums s (facet order)."""
    s = np.empty(h.n, dtype=np.float64)
    _check(_lib.rad_htree_close_cavity(h.ptr, s.ctypes.data, _stream(stream)))
    return s


def rad_htree_set_product_path(h: HTree, path: int) -> None:
    """0: CUDA-core tiles, 1: tensor cores (BF16 x 3 split; the default after
    compression for FP32 / BF16 operators) for >= 5 FP32 columns."""
    _check(_lib.rad_htree_set_product_path(h.ptr, int(path)))


def rad_htree_set_one_column_path(h: HTree, path: int) -> None:
    """One-column product: 1 one fused launch, 0 two launches."""
    _check(_lib.rad_htree_set_one_column_path(h.ptr, int(path)))


def rad_htree_get_stats(h: HTree) -> dict:
    s = _Stats()
    _check(_lib.rad_htree_get_stats(h.ptr, C.byref(s)))
    return {k: getattr(s, k) for k, _ in _Stats._fields_}


def rad_htree_export_tree(h: HTree) -> dict:
    st = rad_htree_get_stats(h)
    nn, n = st["n_nodes"], st["n"]
    out = dict(perm=np.empty(n, np.int32), begin=np.empty(nn, np.int32), end=np.empty(nn, np.int32),
               level=np.empty(nn, np.int32), child=np.empty((nn, 2), np.int32), bbox=np.empty((nn, 6)))
    _check(_lib.rad_htree_export_tree(h.ptr, *(C.c_void_p(out[k].ctypes.data) for k in
                                                ("perm", "begin", "end", "level", "child", "bbox"))))
    return out


def rad_htree_export_blocks(h: HTree) -> dict:
    nb = rad_htree_get_stats(h)["n_blocks"]
    out = {k: np.empty(nb, np.int32) for k in ("row_node", "col_node", "admissible", "rank")}
    _check(_lib.rad_htree_export_blocks(h.ptr, *(C.c_void_p(out[k].ctypes.data) for k in
                                                  ("row_node", "col_node", "admissible", "rank"))))
    return out


def rad_htree_export_block(h: HTree, b: int, m: int, n: int, rank: int):
    """Stored block ``b`` (export order): D (m, n) if dense, else (U, V)."""
    if rank < 0:
        D = np.empty((m, n))
        _check(_lib.rad_htree_export_block(h.ptr, int(b), C.c_void_p(D.ctypes.data), None, None))
        return D
    U = np.zeros((m, max(rank, 0)))
    V = np.zeros((n, max(rank, 0)))
    _check(_lib.rad_htree_export_block(h.ptr, int(b), None, C.c_void_p(U.ctypes.data) if rank else None,
                                       C.c_void_p(V.ctypes.data) if rank else None))
    return U, V


def rad_htree_save(h: HTree) -> bytes:
    """Checkpoint of the handle (trees, compressed operator, work lists)."""
    size = C.c_uint64(0)
    _check(_lib.rad_htree_save(h.ptr, None, C.byref(size)))
    buf = C.create_string_buffer(size.value)
    _check(_lib.rad_htree_save(h.ptr, buf, C.byref(size)))
    return buf.raw[:size.value]


def rad_htree_load(blob: bytes, stream=None, allocator: Allocator | None = None) -> HTree:
    """A handle identical to the one ``blob`` was saved from, on the current device."""
    data = bytes(blob)
    out = C.c_void_p()
    p = _tree_params(1, 1.0, allocator)
    _check(_lib.rad_htree_load(data, len(data), C.byref(p), _stream(stream), C.byref(out)))
    n = int(np.frombuffer(data[12 + 8:12 + 16], dtype=np.int64)[0])
    return HTree(out.value, n, allocator)


def rad_htree_free(h: HTree) -> None:
    h.free()


def rad_launch_count() -> int:
    """Kernels launched by librad in this process."""
    return int(_lib.rad_launch_count())


def rad_profile_enable(on: bool = True) -> None:
    """Start (clearing the record) or stop per-kernel CUDA-event timing."""
    _check(_lib.rad_profile_enable(1 if on else 0))


def rad_profile_read(max_kernels: int = 64) -> dict:
    """{kernel name: (launches, total ms)} of the profile record."""
    names = C.create_string_buffer(48 * max_kernels)
    counts = np.zeros(max_kernels, np.int64)
    ms = np.zeros(max_kernels, np.float64)
    k = _lib.rad_profile_read(max_kernels, names, C.c_void_p(counts.ctypes.data), C.c_void_p(ms.ctypes.data))
    out = {}
    for i in range(min(k, max_kernels)):
        nm = names.raw[48 * i:48 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(counts[i]), float(ms[i]))
    return out


__all__ = [n for n in dir() if n.startswith("rad_")] + ["HTree", "Server", "RadError", "SIGMA_SB",
                                                          "header_functions"]
