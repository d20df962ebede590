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


NAMES = ["warp", "block", "dense", "wdense", "sparse", "wsparse", "hubpair"]


def work(rows=0, w=0, inc=0, pairs=0, nonhub=0, scan_c=0, scan_f=0):
    return [rows, w, inc, pairs, nonhub, scan_c, scan_f]


def mode_work_of(per_list):
    """per_list[s] = {handler name: work(...)}; other handlers do nothing."""
    return {s: [per_list[s].get(n, work()) for n in NAMES] for s in per_list}


def cand(cands, pas, name):
    return next(c for c in cands if c[0] == pas and c[1] == NAMES.index(name))


def zero_times():
    return [[1.0] * len(NAMES), [1.0] * len(NAMES)], [[1] * len(NAMES), [1] * len(NAMES)]


def test_walk_candidates_one_walk_windows():
    # one-walk windows: the hub-pair counting pass walks list 0's plan once and
    # stages its pairs (5 B each); its fill pass is not charged; list 4 is
    # filtered, so nothing of it is charged to the walks
    mw = mode_work_of({2: {"hubpair": work(w=1000, inc=10, pairs=100, nonhub=300)},
                       4: {"hubpair": work(w=1000, inc=10, pairs=7, nonhub=300)}})
    made = {2: [3, 100, 0, 0, 0, 0], 4: [0, 0, 3, 7, 5, 100]}
    ms, ln = zero_times()
    cands, one_walk, walk_f = bench.walk_candidates(NAMES, mw, [2, 4], "stream", made, ms, ln, 1)
    assert cand(cands, "count", "hubpair")[2] == 4 * 300 + 8 * 10 + 5 * 100
    assert cand(cands, "fill", "hubpair")[2] == 0
    assert walk_f == {2: 1.0, 4: 0.0}
    assert all(one_walk(k) for k in range(len(NAMES)))


def test_walk_candidates_ensemble_filter_and_per_s():
    # an ensemble in windows of every list: one counting walk of the sparse
    # accumulator for both lists; list 2 walked in every window, list 3 in half
    # of them (its pairs split the same way between fill and filter)
    mw = mode_work_of({2: {"sparse": work(w=800, inc=20, pairs=50)},
                       3: {"sparse": work(w=800, inc=20, pairs=20)}})
    made = {2: [4, 50, 0, 0, 0, 0], 3: [2, 12, 2, 8, 1, 30]}
    ms, ln = zero_times()
    cands, _, walk_f = bench.walk_candidates(NAMES, mw, [2, 3], "ensemble", made, ms, ln, 1)
    assert cand(cands, "count", "sparse")[2] == 4 * 800 + 8 * 20
    walk = 4 * 800 + 8 * 20
    assert cand(cands, "fill", "sparse")[2] == walk * (1 + 0.5) + 12 * (50 + 20 * 12 / 20)
    assert walk_f == {2: 1.0, 3: 0.5}
    # one s at a time: every list counted and filled by its own walk
    cands, one_walk, _ = bench.walk_candidates(NAMES, mw, [2, 3], "per_s", {}, ms, ln, 2)
    assert cand(cands, "count", "sparse")[2] == 2 * walk
    assert cand(cands, "fill", "sparse")[2] == 2 * walk + 12 * 70
    assert cand(cands, "fill", "sparse")[3] == 0.5  # ms per step over 2 steps
    assert not any(one_walk(k) for k in range(len(NAMES)))


def test_walk_candidates_dense_bytes():
    # dense handlers: non-hub wedges, one hub mask per scanned partner, bounds
    mw = mode_work_of({1: {"wdense": work(w=10**6, inc=40, pairs=900, nonhub=15000, scan_c=3000,
                                          scan_f=2500)}})
    ms, ln = zero_times()
    cands, _, _ = bench.walk_candidates(NAMES, mw, [1], "ensemble", {}, ms, ln, 1)
    assert cand(cands, "count", "wdense")[2] == 4 * 15000 + 4 * 3000 + 8 * 40
    assert cand(cands, "fill", "wdense")[2] == 4 * 15000 + 4 * 2500 + 8 * 40 + 12 * 900
    assert cand(cands, "fill", "wdense")[5] == 4 * 10**6 + 8 * 40 + 12 * 900


def test_default_sweeps():
    assert bench.sweep_of(args(sweep=None, ens_windows=None)) == ("ensemble", False)
    assert bench.sweep_of(args(workload="large", sweep=None, ens_windows=None)) == ("stream", True)
    assert bench.sweep_of(args(sweep="per_s", ens_windows="all")) == ("per_s", True)
    assert bench.sweep_of(args(workload="large", sweep="ensemble", ens_windows="per_list")) == \
        ("ensemble", False)
