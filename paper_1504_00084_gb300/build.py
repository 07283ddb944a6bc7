"""In-tree build of the SDD CUDA library (libsdd.so) for sm_103a.

Each translation unit is compiled in parallel with nvcc, then linked into
paper_1504_00084_gb300/_build/libsdd.so (git-ignored).  No cmake, one -gencode.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libsdd.so")
SOURCES = ["sdd_api.cu", "sdd_prep.cu", "sdd_mc.cu", "sdd_solve.cu", "sdd_noalloc.cu", "sdd_batch.cu",
           "sdd_server.cu"]
HEADERS = [os.path.join(CSRC, "sdd_internal.cuh"), os.path.join(CSRC, "sdd_problem.cuh"),
           os.path.join(ROOT, "include", "sdd.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def flags(extra=()):
    return ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]


CHECKED = os.path.join(BUILD, "checked")  # -DSDD_BOUNDS_CHECK build (test use)
SANITIZED = os.path.join(BUILD, "asan")   # host code under AddressSanitizer + UBSan (test use)
SAN_FLAGS = "-fsanitize=address,-fsanitize=undefined,-fno-omit-frame-pointer"


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in [src, *HEADERS])


def build(force: bool = False, verbose_ptxas: bool = False, bounds_check: bool = False,
          sanitize: bool = False) -> str:
    """Compile and link the library.  bounds_check builds the index-checked variant into
    _build/checked/libsdd.so; sanitize builds one whose host code carries AddressSanitizer and
    UBSan into _build/asan/libsdd.so (load it with libasan preloaded)."""
    out_dir = CHECKED if bounds_check else (SANITIZED if sanitize else BUILD)
    lib_path = os.path.join(out_dir, "libsdd.so")
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    extra = (["-Xptxas", "-v"] if verbose_ptxas else []) + (["-DSDD_BOUNDS_CHECK"] if bounds_check else [])
    if sanitize:
        extra += ["-Xcompiler", SAN_FLAGS]
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(out_dir, s.replace(".cu", ".o"))
        objs.append(obj)
        if force or verbose_ptxas or _stale(obj, src):
            jobs.append([cc, *flags(extra), "-c", src, "-o", obj])
    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose_ptxas or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    if force or jobs or not os.path.exists(lib_path):
        tmp = lib_path + f".tmp{os.getpid()}"
        link = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart",
                *(["-Xcompiler", SAN_FLAGS] if sanitize else [])]
        r = subprocess.run(link, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv,
                bounds_check="--bounds-check" in sys.argv))
