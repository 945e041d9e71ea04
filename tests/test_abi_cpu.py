"""The C-ABI library builds, loads and exports every symbol include/tcgemm.h declares.

No GPU needed: only host-side argument validation is exercised (it answers
before any device is touched).
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tcgemm.h")
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


def _declared_functions():
    text = "\n".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


@pytest.fixture(scope="module")
def lib():
    from paper_1803_04014_gb300 import binding
    return binding.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("gemm_mixed", "gemm_split", "gemm_grouped", "serve_submit", "serve_poll", "tc_quantize",
                 "tc_error_norm", "gemm_batched_strided", "gemm_sgemm"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1803_04014_gb300 import binding
    names = _declared_functions()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(binding.SIGNATURES), set(names) ^ set(binding.SIGNATURES)
    out = subprocess.run(["nm", "-D", "--defined-only", binding.library_path()], capture_output=True, text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    assert set(names) <= exported


def test_struct_layouts_match_header(tmp_path):
    from paper_1803_04014_gb300 import binding
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "tcgemm.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(tc_problem), sizeof(tc_serve_cfg),"
        " sizeof(tc_request), sizeof(tc_result), offsetof(tc_problem, off_c), offsetof(tc_request, C),"
        " offsetof(tc_request, alpha), sizeof(tc_quantize_job), offsetof(tc_quantize_job, dst),"
        " offsetof(tc_quantize_job, transpose)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(binding.tc_problem), ctypes.sizeof(binding.tc_serve_cfg), ctypes.sizeof(binding.tc_request),
            ctypes.sizeof(binding.tc_result), binding.tc_problem.off_c.offset, binding.tc_request.C.offset,
            binding.tc_request.alpha.offset, ctypes.sizeof(binding.tc_quantize_job), binding.tc_quantize_job.dst.offset,
            binding.tc_quantize_job.transpose.offset]
    assert got == want


def test_version_and_error_string(lib):
    from paper_1803_04014_gb300 import binding
    assert "sm_103a" in binding.tc_version()
    assert isinstance(binding.tc_last_error(), str)


def test_host_validation_without_gpu(lib):
    from paper_1803_04014_gb300 import binding as b
    cases = [
        lambda: lib.gemm_mixed(7, 8, 8, 8, 1.0, None, 8, 0, None, 8, 1, 0.0, None, 8, None, None, None),
        lambda: lib.gemm_mixed(0, -1, 8, 8, 1.0, None, 8, 0, None, 8, 1, 0.0, None, 8, None, None, None),
        lambda: lib.gemm_mixed(0, 8, 8, 8, 1.0, None, 8, 5, None, 8, 1, 0.0, None, 8, None, None, None),
        # more output tiles than the kernels count in 32 bits
        lambda: lib.gemm_mixed(0, 1 << 30, 1 << 30, 8, 1.0, None, 8, 0, None, 8, 1, 0.0, None, 1 << 30, None, None,
                               None),
        lambda: lib.gemm_split(2, 3, 8, 8, 8, 1.0, None, 8, 0, None, 8, 0, 0.0, None, 8, None, 0, None),
        lambda: lib.gemm_split(0, 5, 8, 8, 8, 1.0, None, 8, 0, None, 8, 0, 0.0, None, 8, None, 0, None),
        # the two-phase refinement: a workspace is required, schemes and product counts are checked
        lambda: lib.gemm_split_prepare(0, 0, 3, 8, 8, 8, None, 8, 0, None, 8, 0, None, 0, None),
        lambda: lib.gemm_split_run(0, 0, 3, 8, 8, 8, 1.0, 0.0, None, 8, None, 0, None),
        lambda: lib.gemm_split_run(2, 0, 6, 8, 8, 8, 1.0, 0.0, None, 8, None, 0, None),
        lambda: lib.gemm_split_run(7, 0, 3, 8, 8, 8, 1.0, 0.0, None, 8, None, 0, None),
        lambda: lib.gemm_split_prepare(1, 0, 4, 8, 8, 8, None, 8, 0, None, 8, 0, None, 0, None),
        lambda: lib.tc_quantize(9, 4, 4, None, 4, None, 4, 0, None, None),
        lambda: lib.tc_quantize(2, 4, 4, None, 4, None, 4, 0, None, None),   # E4M3 without a scale word
        lambda: lib.tc_split(2, 4, 4, None, 4, 0, None, None, 4, None),
        lambda: lib.gemm_batched_strided(2, 10, 16, 16, 16, 1.0, None, 256, 0, None, 256, 0, 0.0, None, 256, None),
        lambda: lib.gemm_batched_strided(0, 10, 32, 16, 16, 1.0, None, 256, 0, None, 256, 0, 0.0, None, 256, None),
    ]
    for f in cases:
        assert f() in (b.TC_ERR_INVALID, b.TC_ERR_UNSUPPORTED)
    # empty problems are no-ops that touch nothing
    assert lib.gemm_mixed(0, 0, 8, 8, 1.0, None, 8, 0, None, 8, 1, 0.0, None, 8, None, None, None) == b.TC_OK
    assert lib.gemm_split_workspace_bytes(0, 3, 100, 50, 30) >= 2 * 2 * (100 + 50) * 30


def test_grouped_plan_rejects_bad_problems(lib):
    from paper_1803_04014_gb300 import binding as b
    plan = ctypes.c_void_p()
    bad = b.problems_array([(16, 16, 16, 0, 0, 0, 12, 16, 16)])          # lda not a multiple of 8
    assert lib.gemm_grouped_plan_create(0, 1, bad, 0, 0, ctypes.byref(plan)) == b.TC_ERR_INVALID
    zero = b.problems_array([(0, 16, 16, 0, 0, 0, 16, 16, 16)])
    assert lib.gemm_grouped_plan_create(0, 1, zero, 0, 0, ctypes.byref(plan)) == b.TC_ERR_INVALID
    assert lib.gemm_grouped_plan_create(2, 1, zero, 0, 0, ctypes.byref(plan)) == b.TC_ERR_UNSUPPORTED
    assert "grouped" in b.tc_last_error()


def test_grouped_workspace_covers_both_kernels(lib):
    # gemm_grouped_ws puts either kernel's data in the caller's workspace: for the tcgen05 kernel
    # two 128-byte tensor maps per problem and a 48-byte record per 128 x 256 tile, for the
    # mma.sync kernel a 48-byte problem entry and a 16-byte record per 64 x 64 tile
    from paper_1803_04014_gb300 import binding as b
    assert lib.gemm_grouped_workspace_bytes(0, None) == 0
    one = b.problems_array([(16, 16, 16, 0, 0, 0, 16, 16, 16)])
    assert lib.gemm_grouped_workspace_bytes(1, one) >= 2 * 128 + 48
    big = b.problems_array([(300, 600, 64, 0, 0, 0, 64, 64, 600)])      # 3 x 3 tcgen05 tiles, 5 x 10 mma.sync tiles
    assert lib.gemm_grouped_workspace_bytes(1, big) >= max(2 * 128 + 9 * 48, 48 + 50 * 16)
    rows = [(16 * (1 + g % 16), 16 * (1 + g % 7), 32, 0, 0, 0, 32, 32, 256) for g in range(1000)]
    sizes = [lib.gemm_grouped_workspace_bytes(c, b.problems_array(rows[:c])) for c in (10, 100, 1000)]
    assert sizes[0] < sizes[1] < sizes[2] and sizes[2] >= 1000 * (2 * 128 + 48)
    # m < n <= 256 runs transposed: n = 200 rows in two 128-row tiles unless they run as one tall
    # tile (TCGEMM_GROUPED_TALL=0 turns those off), so the size must cover two
    wide = b.problems_array([(16, 200, 32, 0, 0, 0, 32, 32, 200)])
    assert lib.gemm_grouped_workspace_bytes(1, wide) >= 2 * 128 + 2 * 48
    many = b.problems_array([(16, 200, 32, 0, 0, 0, 32, 32, 200)] * 100)
    assert lib.gemm_grouped_workspace_bytes(100, many) >= 100 * (2 * 128 + 2 * 48)
    # a workspace that is not a 256-byte aligned device pointer is refused before any device work
    st = lib.gemm_grouped_ws(0, 1, one, ctypes.c_void_p(256), 0, ctypes.c_void_p(256), 0, ctypes.c_void_p(256),
                             1.0, 0.0, None, 1 << 20, None)
    assert st == b.TC_ERR_INVALID and "workspace" in b.tc_last_error()


def test_serve_rejects_bad_config(lib):
    from paper_1803_04014_gb300 import binding as b
    cfg = b.tc_serve_cfg(0, 4, 2, 16, 0)
    srv = ctypes.c_void_p()
    assert lib.serve_open(ctypes.byref(cfg), ctypes.byref(srv)) == b.TC_ERR_INVALID
    assert lib.serve_poll(None, 1, None) == b.TC_ERR_INVALID


def test_autotune_table_save_and_load(lib, tmp_path):
    from paper_1803_04014_gb300 import binding as b
    good = tmp_path / "tune.txt"
    # lines of the current format (pair, group_m, tail, korder, cluster, bn), of the ten-field
    # format without bn (read as bn = 256) and of the older seven-field format (tail = 1,
    # korder = 1, cluster = 2, bn = 256)
    good.write_text("# comment\n0 13 13 13 1 16 0 1 4 256 0.65\n1 10 10 10 0 8 0.01\n2 12 12 12 1 4 1 0 2 0.2\n"
                    "0 8 8 8 0 8 1 1 2 64 0.004\n0 11 11 11 1 8 2 1 2 256 0.1\n")
    b.tc_autotune_load(good)
    out = tmp_path / "out.txt"
    b.tc_autotune_save(out)
    lines = [l for l in out.read_text().splitlines() if not l.startswith("#")]
    assert any(l.startswith("0 13 13 13 1 16 0 1 4 256 ") for l in lines)
    assert any(l.startswith("1 10 10 10 0 8 1 1 2 256 ") for l in lines)
    assert any(l.startswith("2 12 12 12 1 4 1 0 2 256 ") for l in lines)
    assert any(l.startswith("0 8 8 8 0 8 1 1 2 64 ") for l in lines)
    assert any(l.startswith("0 11 11 11 1 8 2 1 2 256 ") for l in lines)   # tail 2: parts of K
    for text in ("0 13 13 13 7 16 0.5\n",               # pair must be 0 or 1
                 "0 13 13 13 1 16 3 1 2 0.5\n",         # tail must be 0, 1 or 2
                 "0 13 13 13 1 16 1 5 2 0.5\n",         # korder must be 0 or 1
                 "0 13 13 13 1 16 1 1 3 0.5\n",         # cluster must be 2 or 4
                 "0 13 13 13 0 16 1 1 2 96 0.5\n",      # bn must be 64, 128 or 256
                 "0 13 13 13 0 16 1 1 2 64 0.5 7\n",    # nothing after the time
                 "0 13 13 x 0 16 1 1 2 64 0.5\n"):      # fields are numbers
        bad = tmp_path / "bad.txt"
        bad.write_text(text)
        with pytest.raises(b.TcError):
            b.tc_autotune_load(bad)
    with pytest.raises(b.TcError):
        b.tc_autotune_load(tmp_path / "missing.txt")
