"""Host-side logic of the benchmark (no GPU): argument parsing, workload choice, and
the use of the committed ncu traffic record."""
import json
import os
import shutil
import types

import bench


def args(**kw):
    base = dict(workload="medium", m=1_000_000, s="1-8", cpu_rows=600)
    base.update(kw)
    return types.SimpleNamespace(**base)


def test_s_values():
    assert bench.s_values("1-8") == list(range(1, 9))
    assert bench.s_values("2,4,8,16") == [2, 4, 8, 16]
    assert bench.s_values("1-3,7") == [1, 2, 3, 7]


def test_large_workload_defaults(monkeypatch):
    made = {}

    def fake_cached(key, make):
        made["key"] = key
        return types.SimpleNamespace(m=20_000_000, n=10_000_000, nnz=1)

    monkeypatch.setattr(bench.synth, "cached", fake_cached)
    h, s_list, text, metric, rows = bench.workload_spec(args(workload="large"))
    assert made["key"] == "large_m20000000_seed0"
    assert s_list == [2, 4, 8, 16] and rows == 40
    assert "large" in metric and "Zipf(1.8)" in text
    # an explicit s list and row sample are kept
    _, s_list, _, _, rows = bench.workload_spec(args(workload="large", s="4", cpu_rows=8))
    assert s_list == [4] and rows == 8


def _copy_sources(tmp_path):
    root = tmp_path / "repo"
    (root / "paper_2201_11326_gb300" / "csrc").mkdir(parents=True)
    (root / "profiles").mkdir()
    for f in ("count_fill.cu", "kernel_util.cuh"):
        shutil.copy(os.path.join(bench.ROOT, "paper_2201_11326_gb300", "csrc", f),
                    root / "paper_2201_11326_gb300" / "csrc" / f)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "traffic.json"), root / "profiles")
    return root


def test_traffic_key_ignores_comments_not_code(tmp_path, monkeypatch):
    root = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    k = "k_wdense_items<1, 0>"
    key0 = bench.kernel_source_sha(k)
    src = root / "paper_2201_11326_gb300" / "csrc" / "count_fill.cu"
    text = src.read_text()
    banner = "// " + "=" * 58 + " MODE_WDENSE"
    src.write_text(text.replace(banner, banner + "\n// a new comment line\n\n", 1))
    assert bench.kernel_source_sha(k) == key0
    a = text.index("constexpr int WD_RING = 256;")
    src.write_text(text[:a] + "constexpr int WD_RING = 128;" + text[a + len("constexpr int WD_RING = 256;"):])
    assert bench.kernel_source_sha(k) != key0


def test_traffic_scaled_by_pairs_and_dropped_on_change(tmp_path, monkeypatch):
    root = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    k = "k_wdense_items<1, 0>"
    rec = json.load(open(root / "profiles" / "traffic.json"))[k]
    rec["source_sha"] = bench.kernel_source_sha(k)
    json.dump({k: rec}, open(root / "profiles" / "traffic.json", "w"))
    got = bench.profiled_traffic(k, alg_bytes_per_launch=1e12, pairs_per_launch=1e9)
    assert got == int(rec["dram_per_pair"] * 1e9)
    assert 11.0 < rec["dram_per_pair"] <= 12.5  # the output's 12 B per pair, give or take
    assert bench.profiled_traffic("k_sparse_items<1>", 1e12, 1e9) is None  # no record
    rec["source_sha"] = "0" * 16
    json.dump({k: rec}, open(root / "profiles" / "traffic.json", "w"))
    assert bench.profiled_traffic(k, 1e12, 1e9) is None
