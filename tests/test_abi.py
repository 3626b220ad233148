"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/rad.h declares.  No compute call: this runs without a GPU."""
import ctypes
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2305_06891_gb300", "librad.so")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2305_06891_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_every_declared_function_is_exported(lib):
    import re
    txt = open(os.path.join(ROOT, "include", "rad.h")).read()
    names = set(re.findall(r"^\s*(?:int|const char\*|void)\s+(rad_\w+)\s*\(", txt, re.M))
    assert {"rad_build_htree", "rad_compress_aca", "rad_hmatvec", "rad_solve_flux"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_version_and_binding_names(lib):
    lib.rad_version.restype = ctypes.c_int
    assert lib.rad_version() >= 10000
    import paper_2305_06891_gb300 as rad
    for n in rad.header_functions():
        assert hasattr(rad, n), n


def test_build_targets_sm103a_only():
    from paper_2305_06891_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_null_arguments_are_rejected_without_touching_the_gpu(lib):
    lib.rad_build_htree.restype = ctypes.c_int
    lib.rad_build_htree.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]
    assert lib.rad_build_htree(8, None, None, None, None) == 1   # RAD_EINVAL
    lib.rad_last_error.restype = ctypes.c_char_p
    assert b"null" in lib.rad_last_error()


def test_server_parameters_are_checked_before_any_cuda_call(lib):
    import paper_2305_06891_gb300 as rad
    with pytest.raises(rad.RadError) as e:
        rad.Server(slots=0)
    assert e.value.code == 1
    with pytest.raises(rad.RadError):
        rad.Server(slots=2, hbm_budget_bytes=0)
