"""Build the CUDA library libhgks.so in-tree with nvcc for sm_103a.

Translation units are compiled in parallel (one nvcc per .cu file) and linked
into ``paper_2304_05572_gb300/_lib/libhgks.so``.  No cmake, no torch extension:
the library exposes the C ABI of ``include/hgks.h`` and is loaded with ctypes.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libhgks.so")
LIB_DEBUG = os.path.join(OUT_DIR, "libhgks_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["hgks_kernels.cu", "hgks_api.cu"]
HEADERS = ["hgks_math.cuh", "hgks_internal.h", "erfcx_table.inc"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Build _lib/libhgks.so, or with debug=True _lib/libhgks_debug.so (every kernel access
    checked against the solver's buffers, HGKS_DEBUG_BOUNDS)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if debug:
        common.append("-DHGKS_DEBUG_BOUNDS")
    lib_path = LIB_DEBUG if debug else LIB
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "hgks.h")]
    objs, jobs = [], []
    for src in SOURCES:
        sp = os.path.join(CSRC, src)
        obj = os.path.join(OUT_DIR, src.replace(".cu", "_debug.o" if debug else ".o"))
        objs.append(obj)
        if force or _stale(obj, [sp] + hdrs):
            cmd = common + ["-c", sp, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    if force or jobs or _stale(lib_path, objs):
        tmp = lib_path + ".tmp.%d" % os.getpid()
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
