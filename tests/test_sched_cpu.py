"""The kernels' schedules, compiled for the host (no GPU).

CTA-pair GEMMs (sched_host.cpp): the output-tile raster is a bijection, the cut of a last round into
two parts of K covers every chunk of every tile once, and the persistent grid's only wait (a tile's
second part waits for its first) always ends, on the nominal grid and on every smaller one.

Grouped GEMM (grouped_sched_host.cpp): every output element of every problem lies in exactly one
tile under each setting (tall tiles, transposed problems), and the tile count the host sizes its
buffers by matches the tiles emitted and stays under the setting-free bound.

Both harnesses include the library's own schedule headers."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _run_harness(tmp_path, source, extra_flags=()):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / os.path.splitext(source)[0]
    b = subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", *extra_flags, "-o", str(exe),
                        os.path.join(HERE, source)], capture_output=True, text=True)
    assert b.returncode == 0, b.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_pair_schedule_invariants(tmp_path):
    _run_harness(tmp_path, "sched_host.cpp")


def test_grouped_schedule_covers_every_output_once(tmp_path):
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("no CUDA headers")
    _run_harness(tmp_path, "grouped_sched_host.cpp",
                 ("-I" + cuda_inc, "-I" + os.path.join(os.path.dirname(HERE), "include")))
