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


def test_binding_structs_match_the_header_layout(tmp_path):
    """Size and field offsets of every struct the binding passes across the
    C ABI, against a C program compiled with the header (gcc)."""
    import ctypes as C
    import shutil
    import subprocess

    import paper_2305_06891_gb300 as rad
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"rad_allocator": rad._Allocator, "rad_tree_params": rad._TreeParams,
               "rad_aca_params": rad._AcaParams, "rad_solve_params": rad._SolveParams,
               "rad_solve_info": rad._SolveInfo, "rad_htree_stats": rad._Stats,
               "rad_server_params": rad._ServerParams, "rad_request_info": rad._RequestInfo,
               "rad_server_stats": rad._ServerStats, "rad_hlu_params": rad._HluParams,
               "rad_hlu_stats": rad._HluStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rad.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_checkpoint_blobs_are_validated_before_any_device_work(lib):
    import paper_2305_06891_gb300 as rad
    for blob in (b"", b"NOTRADHT" + bytes(64), b"RADHTREE" + (7).to_bytes(4, "little") + bytes(64),
                 b"RADHTREE" + (1).to_bytes(4, "little") + (10 ** 9).to_bytes(8, "little")):
        with pytest.raises(rad.RadError) as e:
            rad.rad_htree_load(blob)
        assert e.value.code == rad.RAD_EINVAL
