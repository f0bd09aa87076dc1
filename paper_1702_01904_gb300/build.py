"""Build libprism.so in-tree for sm_103a (nvcc for the kernels, g++ for the host engine).

Usage: ``python -m paper_1702_01904_gb300.build [--force] [--verbose]``.
Objects go to ``paper_1702_01904_gb300/_build`` and the library to
``paper_1702_01904_gb300/libprism.so``; both are git-ignored.  The translation units compile
in parallel; a unit is rebuilt only when it or a header is newer than its object.
"""
from __future__ import annotations

import argparse
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libprism.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
HEADERS = [os.path.join(CSRC, h) for h in ("fft.cuh", "params.h", "internal.h", "tc.cuh", "scan_common.cuh", "pass_kernels.cuh",
                                           "tune_shapes.cuh", "tune_pass.cuh", "scan_gemm.cuh", "scan_tc.cuh",
                                           "pass_default.cuh")] + \
    [os.path.join(INCLUDE, "prism.h")]
CUDA_UNITS = ["kernels_build.cu", "kernels_pass_512.cu", "kernels_pass_1024.cu", "kernels_pass_2048.cu", "kernels_tune.cu",
              "kernels_tune_256.cu", "kernels_tune_512_row.cu", "kernels_tune_512_col.cu", "kernels_tune_1024_row.cu",
              "kernels_tune_1024_col.cu", "kernels_tune_2048_row.cu", "kernels_tune_2048_col.cu", "kernels_scan.cu",
              "kernels_tune_scan.cu", "kernels_tc.cu", "kernels_tc_tune.cu", "noalloc.cu"]
HOST_UNITS = ["engine.cpp", "server.cpp"]


def cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _stale(src: str, obj: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + HEADERS)


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build step failed ({r.returncode}): {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr, flush=True)
    return r


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I", INCLUDE, "-I", CSRC]
    jobs = []
    objs = []
    for u in CUDA_UNITS:
        src, obj = os.path.join(CSRC, u), os.path.join(BUILD, u + ".o")
        objs.append(obj)
        if force or _stale(src, obj):
            # every unit's device code compressed in its fatbinary (by default only the larger ones are):
            # the library is about a fifth of the size, and the driver decompresses a module when it loads it
            cmd = [nvcc, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xfatbin=-compress-all", "-Xcompiler", "-fPIC", *inc, "-c",
                   src, "-o", obj]
            if ptxas_verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    for u in HOST_UNITS:
        src, obj = os.path.join(CSRC, u), os.path.join(BUILD, u + ".o")
        objs.append(obj)
        if force or _stale(src, obj):
            jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall", "-pthread",
                         "-I", os.path.join(home, "include"), *inc, "-c", src, "-o", obj])
    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            for f in [ex.submit(_run, j, verbose) for j in jobs]:
                f.result()
    if jobs or force or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + ".tmp"
        _run([nvcc, *ARCH, "-shared", "-cudart", "static", "-Xcompiler", "-pthread", "-o", tmp, *objs], verbose)
        os.replace(tmp, LIB)
    return LIB


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--ptxas", action="store_true", help="print ptxas register/spill report")
    a = ap.parse_args(argv)
    print(build(force=a.force, verbose=a.verbose, ptxas_verbose=a.ptxas))


if __name__ == "__main__":
    sys.exit(main())
