"""Build libspotlight.so in-tree (paper_2606_27262_gb300/_build/).

CUDA sources are compiled for sm_103a only; host sources with g++.  The
translation units compile in parallel and are linked by nvcc (static CUDA
runtime).  Usage: ``python -m paper_2606_27262_gb300.build`` or
``build()`` from Python.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libspotlight.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", *ARCH, "-I", os.path.join(ROOT, "include")]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math"]

CUDA_SOURCES = ["dedisperse.cu", "sps.cu", "sps_noalloc.cu", "probe.cu", "cnn.cu", "cnn_tc.cu", "inject.cu"]
CXX_SOURCES = ["plan.cpp", "capi.cpp", "autotune.cpp", "batch.cpp", "stream.cpp", "sifter.cpp", "cnn.cpp"]


def cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found")


def _sources():
    return [os.path.join(CSRC, s) for s in CUDA_SOURCES + CXX_SOURCES] + [
        os.path.join(CSRC, "sp_internal.h"), os.path.join(CSRC, "sp_cnn_internal.h"), os.path.join(ROOT, "include", "spotlight.h"),
        os.path.join(ROOT, "include", "spotlight_probe.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    inc = ["-I", os.path.join(home, "include"), "-I", os.path.join(ROOT, "include")]
    procs, objs = [], []
    for s in CUDA_SOURCES:
        o = os.path.join(BUILD, s + ".o")
        extra = ["-Xptxas", "-v"] if ptxas_verbose else []
        cmd = [nvcc, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, s), "-o", o]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        objs.append(o)
    for s in CXX_SOURCES:
        o = os.path.join(BUILD, s + ".o")
        cmd = ["g++", *CXX_FLAGS, *inc, "-c", os.path.join(CSRC, s), "-o", o]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        objs.append(o)
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or ptxas_verbose or p.returncode:
            sys.stderr.write(out)
        if p.returncode:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("compile failed:\n" + "\n".join(failed))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, "-shared", *ARCH, "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_verbose="--ptxas" in sys.argv)
    print(LIB)
