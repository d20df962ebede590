"""The no-allocation scan entry point against the library's regular path.

slg_scan_counts_noalloc serves callers that cannot allocate device memory
(their HBM is reserved by another allocator, or cudaMalloc's possible device
synchronisation is not acceptable on their path). It turns per-row pair counts
into list offsets using a fixed array compiled into the library. Here its
output must equal the row offsets that slg_row_offsets computes through the
regular, allocating path, on consecutive calls that reuse the shared array.

This file is collected last on purpose: if it fails, a run stopped at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth
import paper_2201_11326_gb300 as slg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    slg.build.build()
    return torch


def regular_offsets(h, s):
    g = slg.slg_load(h.off, h.idx, h.m, h.n)
    try:
        return slg.slg_row_offsets(g, s)
    finally:
        g.free()


def noalloc_offsets(torch, rowoff, stream):
    counts = torch.from_numpy(np.diff(rowoff).astype(np.int32)).cuda()
    out = torch.full((counts.numel() + 1,), -7, dtype=torch.int64, device="cuda")
    code = slg.lib().slg_scan_counts_noalloc(counts.data_ptr(), out.data_ptr(), counts.numel(),
                                            stream.cuda_stream)
    assert code == slg.SLG_OK, slg.lib().slg_last_error()
    stream.synchronize()
    return out.cpu().numpy()


def one_vertex_rows(m, n):
    # row i = {i mod n}: every row pairs with the later rows sharing its vertex
    off = np.arange(m + 1, dtype=np.int32)
    idx = (np.arange(m) % n).astype(np.int32)
    return synth.Hypergraph(off, idx, n, "one_vertex_rows")


def test_noalloc_scan_equals_regular_path(torch_cuda):
    torch = torch_cuda
    st = torch.cuda.Stream()
    small = synth.medium(seed=11, m=20000)
    big = one_vertex_rows(5_000_000, 5000)   # 2442 level-1 tiles: two-level tile sums
    cases = [(small, 1), (big, 1), (small, 3)]
    for h, s in cases:                        # consecutive calls share the array
        want = regular_offsets(h, s)
        got = noalloc_offsets(torch, want, st)
        assert np.array_equal(got, want), (h.name, s)


def scan_with_noalloc(torch, counts, stream):
    out = torch.full((counts.numel() + 1,), -7, dtype=torch.int64, device="cuda")
    code = slg.lib().slg_scan_counts_noalloc(counts.data_ptr(), out.data_ptr(), counts.numel(),
                                            stream.cuda_stream)
    assert code == slg.SLG_OK, slg.lib().slg_last_error()
    stream.synchronize()
    return out


def test_noalloc_scan_single_tile_and_capacity_edge(torch_cuda):
    # one tile (n <= 2048: no tile sums at all) and exactly the capacity
    # (67,108,864 counts: 32768 level-1 and 16 level-2 tile sums, the last one
    # at the end of the fixed array), against numpy's cumulative sum
    torch = torch_cuda
    st = torch.cuda.Stream()
    rng = np.random.default_rng(31)
    for n in (1, 5, 2047, 2048, 2049, 67_108_864):
        c = rng.integers(0, 4, size=n, dtype=np.int32)
        if n == 67_108_864:
            c[-1] = 1_000_000  # the last count reaches only the last offset
        got = scan_with_noalloc(torch, torch.from_numpy(c).cuda(), st).cpu().numpy()
        want = np.zeros(n + 1, np.int64)
        np.cumsum(c, out=want[1:])
        assert np.array_equal(got, want), n
        del c, got, want


def test_noalloc_scan_allocates_nothing(torch_cuda):
    # after the first call (which may load the library's kernels), further calls
    # change neither torch's allocations nor the device's free memory
    torch = torch_cuda
    st = torch.cuda.Stream()
    counts = torch.randint(0, 9, (3_000_000,), dtype=torch.int32, device="cuda")
    out = torch.empty(counts.numel() + 1, dtype=torch.int64, device="cuda")
    lib = slg.lib()

    def call():
        assert lib.slg_scan_counts_noalloc(counts.data_ptr(), out.data_ptr(), counts.numel(),
                                           st.cuda_stream) == slg.SLG_OK
        st.synchronize()

    call()
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0, (free0, free1)
    want = torch.zeros_like(out)
    want[1:] = torch.cumsum(counts.to(torch.int64), 0)
    assert torch.equal(out, want)


def test_noalloc_scan_limits(torch_cuda):
    torch = torch_cuda
    lib = slg.lib()
    dev = torch.zeros(4, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int32, device="cuda")
    # above the fixed capacity: rejected before any launch
    assert lib.slg_scan_counts_noalloc(cnt.data_ptr(), dev.data_ptr(), 67108865, None) == \
        slg.SLG_EINVAL
    assert b"67108864" in lib.slg_last_error()
    # host memory is refused (the call may not stage through new buffers)
    host = np.zeros(5, np.int64)
    assert lib.slg_scan_counts_noalloc(cnt.data_ptr(), host.ctypes.data, 4, None) == \
        slg.SLG_EINVAL
    # n = 0 writes offsets[0] = 0
    dev.fill_(5)
    assert lib.slg_scan_counts_noalloc(None, dev.data_ptr(), 0, None) == slg.SLG_OK
    torch.cuda.synchronize()
    assert int(dev[0]) == 0
