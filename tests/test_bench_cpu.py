"""Host logic of bench.py that decides what its JSON line claims: which kernel configuration the
headline GEMM runs in, which kernel that is, and whether the committed ncu summary's DRAM traffic
may be reported for it (only for the kernel source and the configuration it was taken of)."""
import os
import re

import bench


def _profile_fields():
    text = open(os.path.join(bench.ROOT, "profiles", "gemm_mixed_f16_n8192.md")).read()
    traffic = float(re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text).group(1))
    sha = re.search(r"kernel_sources_sha256:\s*([0-9a-f]+)", text).group(1)
    cfg = dict(kv.split("=") for kv in re.search(r"kernel_config:\s*(.+)", text).group(1).split())
    return traffic, sha, cfg


def test_headline_config_from_the_tune_table():
    # no table: the untuned configuration; a table row for FP16 with eleven fields: its fields
    assert bench.headline_config([]) == bench.DEFAULT_GEMM_CFG
    row = ["0", "13", "13", "13", "1", "16", "0", "0", "4", "256", "0.61"]
    assert bench.headline_config([row]) == {"pair": 1, "group_m": 16, "tail": 0, "korder": 0, "cluster": 4,
                                            "bn": 256}
    single = ["0", "13", "13", "13", "0", "8", "1", "1", "2", "64", "0.7"]
    assert bench.headline_config([single])["bn"] == 64
    # rows of other dtypes or of another width are not the headline's
    assert bench.headline_config([["1"] + row[1:]]) == bench.DEFAULT_GEMM_CFG
    assert bench.headline_config([row[:10]]) == bench.DEFAULT_GEMM_CFG


def test_kernel_names_follow_the_configuration():
    assert bench.kernel_name(bench.DEFAULT_GEMM_CFG).startswith("k_tc_gemm_pair")
    assert bench.kernel_name(dict(bench.DEFAULT_GEMM_CFG, cluster=4)).startswith("k_tc_gemm_quad")
    assert "128x64" in bench.kernel_name(dict(bench.DEFAULT_GEMM_CFG, pair=0, bn=64))


def test_traffic_only_for_the_profiled_source_and_configuration(monkeypatch):
    traffic, sha, cfg = _profile_fields()
    prof_cfg = {k: int(v) for k, v in cfg.items()}
    monkeypatch.setattr(bench, "kernel_sources_sha", lambda: sha)
    assert bench.profiled_traffic(prof_cfg) == traffic
    # another configuration or another kernel source: no figure
    assert bench.profiled_traffic(dict(prof_cfg, korder=1 - prof_cfg["korder"])) is None
    monkeypatch.setattr(bench, "kernel_sources_sha", lambda: "0" * 16)
    assert bench.profiled_traffic(prof_cfg) is None


def test_the_profile_was_taken_of_the_untuned_configuration():
    _, _, cfg = _profile_fields()
    assert {k: int(v) for k, v in cfg.items()} == bench.DEFAULT_GEMM_CFG


def test_reference_arm_prints_one_contract_line():
    # the oracle arm runs on the host cores alone: one JSON line with the keys every bench line
    # carries, its cpu_baseline describing this run, and no host<->device bytes
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["higher_is_better"] is True and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    # no CPU fallback: without the built library the binding raises instead of computing anything
    import pytest
    from paper_1803_04014_gb300 import binding, builder
    monkeypatch.setattr(binding, "_LIB", None)
    monkeypatch.setattr(builder, "LIB", str(tmp_path / "libtcgemm.so"))
    with pytest.raises(ImportError):
        binding.load(build_if_needed=False)
