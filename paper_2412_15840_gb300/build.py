"""Build libsylv.so in-tree for sm_103a.

    python -m paper_2412_15840_gb300.build [--force] [--debug]

Translation units compiled in parallel (nvcc for the CUDA sources, the
host C++ Schur code through nvcc's host compiler), one -gencode, static
cudart, linked into paper_2412_15840_gb300/libsylv.so.  No cmake.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libsylv.so")
BUILD = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["kernels.cu", "sweep.cu", "modeprod_tc.cu", "modeprod_tcw.cu", "modeprod_fib.cu", "resid_oz.cu", "real.cu", "capi.cu", "schur.cpp",
           "schur_real.cpp", "expm.cpp"]
HEADERS = ["sylv_internal.h", "cplx.cuh", "tc_ptx.cuh", "sweep_common.cuh", os.path.join("..", "..", "include", "sylv.h")]


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _stale(force: bool) -> bool:
    if force or not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, h) for h in HEADERS]
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, debug: bool = False, verbose: bool = False) -> str:
    if not _stale(force):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    opt = ["-O0", "-g", "-G"] if debug else ["-O3", "-lineinfo"]
    common = ["-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    procs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s + ".o")
        objs.append(obj)
        if s.endswith(".cu"):
            cmd = [nvcc, *ARCH, *opt, *common, "-c", src, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
        else:
            cmd = [nvcc, "-x", "c++", "-O2", *common, "-c", src, "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, pr in procs:
        out, _ = pr.communicate()
        text = out.decode(errors="replace")
        if pr.returncode != 0:
            failed.append((cmd, text))
        elif verbose and text.strip():
            print(text)
    if failed:
        msg = "\n\n".join(" ".join(c) + "\n" + t for c, t in failed)
        raise RuntimeError("libsylv build failed:\n" + msg)
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, *ARCH, "-shared", "-cudart", "static", *objs, "-o", tmp]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("libsylv link failed:\n" + " ".join(link) + "\n" + r.stdout.decode())
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, debug="--debug" in sys.argv,
                verbose="-v" in sys.argv))
