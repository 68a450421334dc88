"""Builds the CUDA library libkfscan.so in-tree for sm_103a with nvcc.

Translation units (one per state dimension plus the C-ABI layer) are
compiled in parallel, then linked into one shared library with the CUDA
runtime linked statically.

build(check=True) makes the bounds-checked variant, _build_check/
libkfscan_check.so (compiled with KF_BOUNDS_CHECK): every index check in the
kernels records KF_ERR_BOUNDS in the status word and skips the access.  It
is a debugging build, selected at import time with the KFSCAN_LIB
environment variable; the product path loads libkfscan.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "_build", "libkfscan.so")
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(BUILD_CHECK, "libkfscan_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = (["kf_api.cu", "kf_serve.cu", "kf_n4_f32_t256.cu", "kf_tv_n2.cu", "kf_tv_n4.cu", "kf_tv_n8.cu",
          "ti_n4_f32.cu", "ti_n2_f32.cu", "ti_n4_f64.cu", "ti_n2_f64.cu", "flop_count.cpp",
          "gain_tables.cpp"]
         + ["gs_n%d_%s.cu" % (n, p) for n in (8, 4, 2) for p in ("f64", "f32")]
         + ["kf_n%d_%s.cu" % (n, p) for n in (8, 4, 2) for p in ("f64", "mix", "f32")]
         + ["kf_n%d_%s_batch.cu" % (n, p) for n, p in ((8, "f64"), (8, "mix"), (8, "f32"), (4, "f64"), (4, "mix"))])


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [
        os.path.join(os.path.dirname(HERE), "include", "kfscan.h")]


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, check: bool = False) -> str:
    lib, bdir = (LIB_CHECK, BUILD_CHECK) if check else (LIB, BUILD)
    if not force and not _stale(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-rdc=false",
                    "--expt-relaxed-constexpr", "-I", os.path.join(os.path.dirname(HERE), "include")]
    if check:
        flags += ["-DKF_BOUNDS_CHECK"]
    if ptxas_info:
        flags += ["-Xptxas", "-v"]

    def compile_one(u):
        src = os.path.join(CSRC, u)
        obj = os.path.join(bdir, os.path.splitext(u)[0] + ".o")
        cmd = [cc, "-c", src, "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (u, r.stdout, r.stderr))
        return obj, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(compile_one, UNITS))
    if verbose or ptxas_info:
        for obj, log in results:
            sys.stderr.write(log)
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [cc, "-shared", "-o", tmp] + [o for o, _ in results] + ARCH + ["-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                check="--check" in sys.argv))
