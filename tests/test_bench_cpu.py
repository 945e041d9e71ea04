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
