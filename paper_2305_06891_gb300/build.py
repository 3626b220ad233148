"""Build librad.so (the CUDA C-ABI library) in-tree for sm_103a.

Usage: python -m paper_2305_06891_gb300.build [--force] [--verbose]

Every ``csrc/*.cu`` file is compiled in parallel with nvcc into ``_build/``
and linked into ``paper_2305_06891_gb300/librad.so``; the same objects with
the allocation layer compiled for bounds checking (canary words around every
device allocation) form ``librad_checked.so``.  Objects are rebuilt when a
source or header is newer than them.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "librad.so")
LIB_CHECKED = os.path.join(PKG, "librad_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librad")
    return cand


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _compile(src: str, force: bool, verbose: bool, extra: list[str], suffix: str = "") -> str:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + suffix + ".o")
    if (not force and os.path.exists(obj)
            and os.path.getmtime(obj) >= max(os.path.getmtime(src), _headers_mtime())):
        return obj
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr, flush=True)
    return obj


def _link(lib: str, objs: list[str], force: bool, verbose: bool) -> None:
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + ".tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64",
               "-o", tmp, *objs]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Builds librad.so and its bounds-checked twin librad_checked.so (the
    allocation layer, api.cu, compiled with RAD_CHECK_BOUNDS; every other
    object shared)."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    api = os.path.join(CSRC, "api.cu")
    jobs = [(s, extra or [], "") for s in srcs] + [(api, (extra or []) + ["-DRAD_CHECK_BOUNDS"], "_checked")]
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        objs = list(ex.map(lambda j: _compile(j[0], force, verbose, j[1], j[2]), jobs))
    plain, checked_api = objs[:-1], objs[-1]
    _link(LIB, plain, force, verbose)
    api_obj = os.path.join(BUILD, "api.o")
    _link(LIB_CHECKED, [checked_api if o == api_obj else o for o in plain], force, verbose)
    return LIB


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    a = ap.parse_args(argv)
    print(build(a.force, a.verbose))
    return 0


if __name__ == "__main__":
    sys.exit(main())
