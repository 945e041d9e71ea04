"""The CTA-pair kernels' schedule, compiled for the host (no GPU): the output-tile raster is a
bijection, the cut of a last round into two parts of K covers every chunk of every tile once, and
the persistent grid's only wait (a tile's second part waits for its first) always ends, on the
nominal grid and on every smaller one.  The checks live in sched_host.cpp, which includes the
kernels' own schedule header."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_pair_schedule_invariants(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "sched_host"
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-o", str(exe),
                    os.path.join(HERE, "sched_host.cpp")], check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
