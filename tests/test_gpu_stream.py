"""One-walk windows (slg_stream_window, slg_ensemble_stream_window).

Windows are chosen from a bound on their rows' pairs before the rows are
walked, and the sparse-accumulator and hub-pair rows are walked once (their
pairs staged, then copied into place). Whatever the handlers, the pool and the
buffer size, consecutive windows must cover the rows once, in order, and their
lists concatenated must equal the oracle's L_s for each threshold, element by
element. A graph whose first rows have many wedges and almost no pairs makes
the second window's estimate fall short, so its list 0 and then its later
lists are cut back to what fits.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2201_11326_gb300 as slg
from tests.test_gpu_parity import FORCED, assert_same
from tests.test_oracle_pins import csr_from_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    slg.build.build()
    return torch


_ORACLE = {}


def oracle_list(key, h, s):
    if (key, s) not in _ORACLE:
        _ORACLE[(key, s)] = oracle.slg_par(h.off, h.idx, s)
    return _ORACLE[(key, s)]


def stream_all(torch, g, s_list, cap):
    """Every window from row 0; per list the concatenated (I, J, O), and the windows."""
    I = torch.empty(cap, dtype=torch.int32, device="cuda")
    J = torch.empty_like(I)
    O = torch.empty_like(I)
    k = len(s_list)
    parts = [[] for _ in range(k)]
    windows = []
    r0 = 0
    while r0 < g.m:
        r1, pairs = slg.slg_ensemble_stream_window(g, s_list, r0, I, J, O, cap)
        assert r0 < r1 <= g.m, (r0, r1)
        assert sum(pairs) <= cap
        hi, hj, ho = I.cpu().numpy(), J.cpu().numpy(), O.cpu().numpy()
        b = 0
        for t, p in enumerate(pairs):
            parts[t].append((hi[b:b + p].copy(), hj[b:b + p].copy(), ho[b:b + p].copy()))
            b += p
        windows.append((r0, r1, pairs))
        r0 = r1
    # past the last row: nothing, and the end stays at m
    assert slg.slg_ensemble_stream_window(g, s_list, g.m, I, J, O, cap) == (g.m, [0] * k)
    lists = [tuple(np.concatenate([p[c] for p in parts[t]]) if parts[t] else
                   np.zeros(0, np.int32) for c in range(3)) for t in range(k)]
    return lists, windows


def check_stream(torch, h, key, s_list, cap, bins=None, hub_pairs=None, staging=None):
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        if bins is not None:
            slg.slg_set_bins(g, *bins)
        if hub_pairs is not None:
            slg.slg_set_hub_pairs(g, *hub_pairs)
        if staging is not None:
            slg.slg_set_staging(g, staging)
        lists, windows = stream_all(torch, g, s_list, cap)
        # the regular calls still agree afterwards (the plan's counts are redone)
        pairs, _ = slg.slg_ensemble_count(g, s_list)
    finally:
        g.free()
    for s, got, p in zip(s_list, lists, pairs):
        want = oracle_list(key, h, s)
        assert p == want[0].size
        assert_same(got, want, f"{key} stream {list(s_list)} s={s} cap={cap} bins={bins}")
    return windows


@pytest.mark.parametrize("handler", ["default", "hubpair", "sparse_cta_only", "block_only"])
@pytest.mark.parametrize("s_list", [[2], [2, 3, 5, 8]])
def test_stream_windows_match_oracle(torch_cuda, handler, s_list):
    h = synth.large(m=20000)
    want = sum(oracle_list("large20000", h, s)[0].size for s in s_list)
    cap = max(want // 9, 4096)
    if handler == "hubpair":
        kw = dict(bins=FORCED["block_only"], hub_pairs=(512, 0))
    else:
        kw = dict(bins=FORCED[handler], hub_pairs=(0, 0))
    windows = check_stream(torch_cuda, h, "large20000", s_list, cap, **kw)
    assert len(windows) >= 9


@pytest.mark.parametrize("pool", ["off", "small"])
def test_stream_windows_with_small_or_no_pool(torch_cuda, pool):
    # no pool: every row walked twice; a small pool (a few hundred thousand
    # pairs): items that do not fit are walked again by the fill
    h = synth.large(m=20000)
    staging = 0 if pool == "off" else 8 * 200000 + 5 * 4096
    want = oracle_list("large20000", h, 2)[0].size
    check_stream(torch_cuda, h, "large20000", [2, 4], max(want // 5, 4096),
                 bins=FORCED["sparse_cta_only"], hub_pairs=(0, 0), staging=staging)


def wedge_heavy_then_pair_heavy():
    """Rows 0..999 share vertex 0 and nothing else (many wedges, one pair:
    rows 0 and 1 are equal); rows 1000..2999 come in groups of ten equal rows
    of 40 fresh vertices (45 pairs a group, overlap 40)."""
    rows, nxt = [], 1
    for i in range(1000):
        if i == 1:
            rows.append(list(rows[0]))
            continue
        rows.append([0] + list(range(nxt, nxt + 39)))
        nxt += 39
    for _ in range(200):
        grp = list(range(nxt, nxt + 40))
        nxt += 40
        rows += [grp] * 10
    off, idx = csr_from_rows(rows)
    return synth.Hypergraph(off, idx, nxt, "wedge_heavy_then_pair_heavy")


@pytest.mark.parametrize("bins", ["default", "sparse_cta_only"])
def test_stream_windows_cut_when_the_estimate_falls_short(torch_cuda, bins):
    h = wedge_heavy_then_pair_heavy()
    for s_list in ([2], [2, 3]):
        windows = check_stream(torch_cuda, h, "wedge_heavy", s_list, 3000, bins=FORCED[bins],
                               hub_pairs=(0, 0))
        # the 9000 pairs of the second part need several windows of 3000
        assert len(windows) >= 3 + len(s_list)
        assert all(sum(p) <= 3000 for _, _, p in windows)


def test_stream_window_errors(torch_cuda):
    torch = torch_cuda
    h = synth.large(m=2000)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    I = torch.empty(4, dtype=torch.int32, device="cuda")
    try:
        with pytest.raises(slg.SlgError):          # a row with more pairs than cap
            r0 = 0
            while r0 < g.m:
                r0, _ = slg.slg_stream_window(g, 1, r0, I, I, I, 4)
        with pytest.raises(slg.SlgError):          # host arrays
            host = np.zeros(16, np.int32)
            slg.slg_stream_window(g, 2, 0, host, host, host, 16)
        for bad in ([3, 2], [0], []):
            with pytest.raises(slg.SlgError):
                slg.slg_ensemble_stream_window(g, bad, 0, I, I, I, 4)
        with pytest.raises(slg.SlgError):
            slg.slg_stream_window(g, 2, g.m + 1, I, I, I, 4)
        with pytest.raises(slg.SlgError):
            slg.slg_stream_window(g, 2, 0, I, I, I, 0)
    finally:
        g.free()
