"""Build the tcgemm shared library in-tree for sm_103a.

nvcc compiles every CUDA translation unit of ``csrc/`` in parallel
(``-gencode arch=compute_103a,code=sm_103a -lineinfo``), g++ compiles the host
scheduler, nvcc links ``_build/libtcgemm.so`` with the static CUDA runtime.
Runs without a GPU (cross-compilation).  Rebuilds only when a source is newer
than the library.
"""
from __future__ import annotations

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
LIB = os.path.join(BUILD, "libtcgemm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.isdir(home):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _nvcc() -> str:
    return os.path.join(_cuda_home(), "bin", "nvcc")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu"))), sorted(glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    cu, cpp = sources()
    return cu + cpp + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(INCLUDE, "tcgemm.h"), os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(verbose: bool = False, extra_nvcc=None) -> str:
    """Compile (if needed) and return the path of libtcgemm.so."""
    if up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cu, cpp = sources()
    nvcc = _nvcc()
    cuda_inc = os.path.join(_cuda_home(), "include")
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-I", CSRC]
    jobs = []
    for src in cu:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-c", src, "-o", obj,
               *common, *(extra_nvcc or [])]
        jobs.append((cmd, obj))
    for src in cpp:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = ["g++", "-fPIC", "-c", src, "-o", obj, "-pthread", "-I", cuda_inc, *common]
        jobs.append((cmd, obj))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        futs = [ex.submit(_run, cmd) for cmd, _ in jobs]
        outs, errs = [], []
        for f in futs:
            try:
                outs.append(f.result())
            except RuntimeError as e:
                errs.append(str(e))
    if errs:
        raise RuntimeError("\n".join(errs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    tmp = LIB + f".{os.getpid()}.tmp"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *[o for _, o in jobs], "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
