"""The row-range sharded product path, run rank after rank on one GPU.

Rows are the independent units of Algorithm 2's parallel loop (Section III-C):
each of four "ranks" builds its row range with slg_build_window, the ranges
are placed by the exclusive prefix of the ranks' pair counts, and the
concatenation must equal the oracle's canonical list. The ranges balance
per-row work from slg_row_offsets (pairs) and the graph's wedge counts.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2201_11326_gb300 as slg
from paper_2201_11326_gb300 import shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    slg.build.build()


def row_wedges(h, s):
    sizes = np.diff(h.off).astype(np.int64)
    row = np.repeat(np.arange(h.m, dtype=np.int64), sizes)
    keep = sizes[row] >= s
    v, r = h.idx[keep].astype(np.int64), row[keep]
    order = np.lexsort((r, v))
    vs, rs = v[order], r[order]
    later = np.searchsorted(vs, vs, side="right") - 1 - np.arange(vs.size)
    w = np.zeros(h.m, np.int64)
    np.add.at(w, rs, later)
    return w


@pytest.mark.parametrize("s", [1, 3])
def test_four_rank_row_ranges_concatenate_to_the_canonical_list(s):
    import torch
    h = synth.medium(seed=13, m=12000)
    want = oracle.slg_par(h.off, h.idx, s)
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        rowoff = slg.slg_row_offsets(g, s)
        work = row_wedges(h, s) + np.diff(rowoff)
        splits = shard.balanced_splits(work, 4)
        assert splits[0] == 0 and splits[-1] == h.m and np.all(np.diff(splits) >= 0)
        parts, counts = [], []
        for r in range(4):  # each rank's slice, into its own device buffers
            r0, r1 = int(splits[r]), int(splits[r + 1])
            n = int(rowoff[r1] - rowoff[r0])
            I = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
            J = torch.empty_like(I)
            O = torch.empty_like(I)
            P, _ = slg.slg_build_window(g, s, r0, r1, I, J, O, max(n, 1))
            assert P == n
            counts.append(P)
            parts.append(tuple(x[:P].cpu().numpy() for x in (I, J, O)))
        base = shard.global_offsets(counts)
        assert base[-1] == want[0].size
        total = int(base[-1])
        got = [np.zeros(total, np.int32) for _ in range(3)]
        for r, p in enumerate(parts):  # placed by the exchanged counts only
            for x in range(3):
                got[x][base[r]:base[r + 1]] = p[x]
        for x in range(3):
            assert np.array_equal(got[x], want[x]), ("IJO"[x], s)
    finally:
        g.free()
