// Per-s planning: pruning to E_s, wedge ranges, per-row work, binning.
//
// Algorithm 2 (Section III-C) skips every e_i with |e_i| < s ("degree-based
// pruning") and, for each kept e_i, visits the wedges (e_i, v_k, e_j) with
// i < j. Pruning e_j as well changes no result (|e_i ∩ e_j| <= |e_j|), so the
// wedge set used here is W_s = { (i, v, j) : i < j, v in e_i ∩ e_j,
// |e_i|, |e_j| >= s }, of size sum_v C(d_s(v), 2) (Section III-E's work).
//
// Instead of relabelling hyperedges by degree and splitting rows into blocked
// or cyclic ranges (Sections III-F and IV), rows are binned by their exact
// wedge count W_{s,i} and candidate span into work items (see slg_internal.cuh),
// so that output ids stay the caller's ids and no un-relabel sort is needed.
#include "slg_internal.cuh"
#include "plan.cuh"

namespace slg {
namespace {

int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

#define GRID_STRIDE(k, n)                                                            \
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < (n);       \
         k += (int64_t)gridDim.x * blockDim.x)

// keep[k] = |e_j| >= s_j for j = idxT[k], for every position k of H^T
__global__ void k_keep_flags(const int32_t* __restrict__ idxT, const int32_t* __restrict__ size,
                             int64_t nnz, RowS rs, int32_t* __restrict__ keep) {
    GRID_STRIDE(k, nnz) {
        const int32_t j = idxT[k];
        keep[k] = size[j] >= rs.s_of(j) ? 1 : 0;
    }
}

// pruned transpose: idxTs[ks[k]] = idxT[k] for kept k (ks = exclusive scan of keep)
__global__ void k_compact(const int32_t* __restrict__ idxT, const int32_t* __restrict__ ks,
                          int64_t nnz, int32_t* __restrict__ idxTs) {
    GRID_STRIDE(k, nnz) {
        const int32_t p = ks[k];
        if (ks[k + 1] != p) idxTs[p] = idxT[k];
    }
}

// Wedge range of incidence e = (i, v): positions of adj_s(v) after i.
__global__ void k_wedge_ranges(const int32_t* __restrict__ idx, const int32_t* __restrict__ rowid,
                               const int32_t* __restrict__ size, const int32_t* __restrict__ tpos,
                               const int32_t* __restrict__ offT, const int32_t* __restrict__ ks,
                               int64_t nnz, RowS rs, int32_t* __restrict__ wbeg,
                               int32_t* __restrict__ wend) {
    GRID_STRIDE(e, nnz) {
        const int32_t i = rowid[e];
        int32_t b = 0, t = 0;
        if (size[i] >= rs.s_of(i)) {
            const int32_t v = idx[e];
            const int32_t p = tpos[e];
            b = (ks ? ks[p] : p) + 1;
            t = ks ? ks[offT[v + 1]] : offT[v + 1];
        }
        wbeg[e] = b;
        wend[e] = t;
    }
}

// One warp per row: W_{s,i} = sum of wedge-range lengths, and the first and
// last candidate j (adj_s lists are ascending, so these are range ends).
__global__ void k_row_work(const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                           const int32_t* __restrict__ hubidx, const int32_t* __restrict__ wbeg,
                           const int32_t* __restrict__ wend, const int32_t* __restrict__ idxTs,
                           int32_t m, int64_t* __restrict__ W, int32_t* __restrict__ jmin,
                           int32_t* __restrict__ jmax, int32_t* __restrict__ nnh,
                           unsigned long long* __restrict__ wtotal) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long acc_total = 0;
    for (int64_t i = warp; i < m; i += nwarps) {
        int64_t w = 0;
        int32_t lo = INT32_MAX, hi = -1, r = 0;
        for (int32_t e = off[i] + lane; e < off[i + 1]; e += 32) {
            const int32_t b = wbeg[e], t = wend[e];
            if (t > b) {
                w += t - b;
                lo = min(lo, idxTs[b]);
                hi = max(hi, idxTs[t - 1]);
                r += hubidx[idx[e]] < 0 ? 1 : 0;
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            w += __shfl_xor_sync(0xffffffffu, w, d);
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
            r += __shfl_xor_sync(0xffffffffu, r, d);
        }
        if (lane == 0) {
            W[i] = w;
            jmin[i] = lo;
            jmax[i] = hi;
            nnh[i] = r;
            acc_total += (unsigned long long)w;
        }
    }
    if (lane == 0 && acc_total) atomicAdd(wtotal, acc_total);
}

// Hub-pair work of row i for s (MODE_HUBPAIR): the wedge range of each of its
// hub-pair incidences in the pruned pair lists, and per row the entries to
// walk (non-HP-hub wedges plus pair-list hits) and their first and last
// partner. Rows outside E_s get empty ranges.
__global__ void k_pair_ranges(const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                              const int32_t* __restrict__ size, const int32_t* __restrict__ wbeg,
                              const int32_t* __restrict__ wend, const int32_t* __restrict__ idxTs,
                              const int32_t* __restrict__ hp_id, const int32_t* __restrict__ off2,
                              const int32_t* __restrict__ idx2, const int32_t* __restrict__ tpos2,
                              const int32_t* __restrict__ offT2, const int32_t* __restrict__ ks2,
                              const int32_t* __restrict__ idxT2s, int32_t m, RowS rs,
                              int32_t* __restrict__ wbeg2, int32_t* __restrict__ wend2,
                              int64_t* __restrict__ Wp, int32_t* __restrict__ lo2,
                              int32_t* __restrict__ hi2) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < m; i += nwarps) {
        const bool kept = size[i] >= rs.s_of((int32_t)i);
        int64_t w = 0;
        int32_t lo = INT32_MAX, hi = -1;
        for (int32_t e = off[i] + lane; e < off[i + 1]; e += 32) {
            const int32_t b = wbeg[e], t = wend[e];
            if (t > b && hp_id[idx[e]] < 0) {
                w += t - b;
                lo = min(lo, idxTs[b]);
                hi = max(hi, idxTs[t - 1]);
            }
        }
        for (int32_t f = off2[i] + lane; f < off2[i + 1]; f += 32) {
            int32_t b = 0, t = 0;
            if (kept) {
                const int32_t key = idx2[f];
                const int32_t q = tpos2[f];
                b = (ks2 ? ks2[q] : q) + 1;
                t = ks2 ? ks2[offT2[key + 1]] : offT2[key + 1];
            }
            wbeg2[f] = b;
            wend2[f] = t;
            if (t > b) {
                w += t - b;
                lo = min(lo, idxT2s[b]);
                hi = max(hi, idxT2s[t - 1]);
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            w += __shfl_xor_sync(0xffffffffu, w, d);
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
        }
        if (lane == 0) {
            // rows with many hub pairs slice poorly: every work item searches
            // every range; they keep the other handlers
            Wp[i] = (off2[i + 1] - off2[i] <= HP_MAXR) ? w : -1;
            lo2[i] = lo;
            hi2[i] = hi;
        }
    }
}

struct RowItems {
    int32_t mode;
    int32_t count;
    int64_t step;    // j width of each item (dense) or 0 (uniform split)
    int32_t lo, hi;  // the partner range the items split
};

// hub-pair inputs of a row (wp < 0: not available)
struct RowHP {
    int64_t wp;
    int32_t lo, hi;
};

__device__ RowItems classify(int64_t w, int32_t lo, int32_t hi, int32_t size, int32_t nnh,
                             int32_t s, BinParams bp, RowHP hp) {
    RowItems r{MODE_WARP, 0, 0, lo, hi};
    if (w <= 0) return r;
    const int64_t span = (int64_t)hi - lo + 1;
    if (w <= bp.warp_max_wedges) {
        r.mode = MODE_WARP;
        r.count = 1;
        return r;
    }
    const bool dense_wanted = bp.dense_min_density >= 0 &&
                              (span <= 4096 || 256 * w >= (int64_t)bp.dense_min_density * span);
    if (dense_wanted && nnh <= bp.wdense_max_ranges) {
        // warp tiles: non-hub counts <= 32, so any row size fits 16-bit counters
        r.mode = MODE_WDENSE;
        r.step = (int64_t)WD_ITEM * bp.dense_item_tiles;
        r.count = (int32_t)((span + r.step - 1) / r.step);
        return r;
    }
    if (dense_wanted && size <= DENSE_MAX_SIZE && size <= DENSE_MAXE) {
        r.mode = MODE_DENSE;
        r.step = (int64_t)DENSE_TILE * bp.dense_item_tiles;
        r.count = (int32_t)((span + r.step - 1) / r.step);
        return r;
    }
    // hub pairs: at s >= 2 the row walks its non-hub wedges and the rows sharing
    // a pair of its hubs, when that is at most half its wedges (no entry at all:
    // no partner can reach an overlap of 2, and the row has no item)
    if (hp.wp >= 0 && s >= 2 && size <= SP_MAX_SIZE && 2 * hp.wp <= w) {
        r.mode = MODE_HUBPAIR;
        if (hp.wp == 0) return r;
        r.lo = hp.lo;
        r.hi = hp.hi;
        const int64_t span2 = (int64_t)hp.hi - hp.lo + 1;
        int64_t k = (hp.wp + HP_ITEM - 1) / HP_ITEM;
        const int64_t kmax = (span2 + 1023) / 1024;
        if (k > kmax) k = kmax;
        if (k < 1) k = 1;
        r.count = (int32_t)k;
        return r;
    }
    const int64_t tiles = (span + SP_TILE - 1) / SP_TILE;
    if (bp.sparse_min_per_tile >= 0 && size <= SP_MAX_SIZE &&
        w >= (int64_t)bp.sparse_min_per_tile * tiles) {
        // uniform j slices of about sparse_item_wedges wedges, at least 1024 ids wide
        // the warp-level accumulator only where its 4096-id tiles stay sparse
        // (below one wedge per 32 ids) and survivors are rare (s >= 2: at s = 1
        // every partner is one, and the CTA's bitmap ranking writes them
        // faster); other rows keep the CTA's wider tiles
        r.mode = (size <= bp.wsparse_max_size && 32 * w < span && s >= 2) ? MODE_WSPARSE
                                                                            : MODE_SPARSE;
        int64_t k = (w + bp.sparse_item_wedges - 1) / bp.sparse_item_wedges;
        const int64_t kmax = (span + 1023) / 1024;
        if (k > kmax) k = kmax;
        if (k < 1) k = 1;
        r.count = (int32_t)k;
        return r;
    }
    r.mode = MODE_BLOCK;
    int64_t k = (w + bp.block_item_wedges - 1) / bp.block_item_wedges;
    if (k > span) k = span;
    if (k < 1) k = 1;
    r.count = (int32_t)k;
    return r;
}

__device__ __forceinline__ RowHP row_hp(const int64_t* Wp, const int32_t* lo2,
                                        const int32_t* hi2, int64_t i) {
    return Wp ? RowHP{Wp[i], lo2[i], hi2[i]} : RowHP{-1, 0, 0};
}

__global__ void k_item_count(const int64_t* __restrict__ W, const int32_t* __restrict__ jmin,
                             const int32_t* __restrict__ jmax, const int32_t* __restrict__ size,
                             const int32_t* __restrict__ nnh, int32_t m, RowS rs, BinParams bp,
                             const int64_t* __restrict__ Wp, const int32_t* __restrict__ lo2,
                             const int32_t* __restrict__ hi2, int32_t* __restrict__ nitem) {
    GRID_STRIDE(i, m) {
        nitem[i] = classify(W[i], jmin[i], jmax[i], size[i], nnh[i], rs.s_of((int32_t)i), bp,
                            row_hp(Wp, lo2, hi2, i)).count;
    }
}

__global__ void k_item_emit(const int64_t* __restrict__ W, const int32_t* __restrict__ jmin,
                            const int32_t* __restrict__ jmax, const int32_t* __restrict__ size,
                            const int32_t* __restrict__ nnh, int32_t m, RowS rs, BinParams bp,
                            const int64_t* __restrict__ Wp, const int32_t* __restrict__ lo2,
                            const int32_t* __restrict__ hi2, const int32_t* __restrict__ row_item,
                            Item* __restrict__ items) {
    GRID_STRIDE(i, m) {
        const RowItems r = classify(W[i], jmin[i], jmax[i], size[i], nnh[i], rs.s_of((int32_t)i), bp,
                                    row_hp(Wp, lo2, hi2, i));
        if (r.count == 0) continue;
        const int64_t lo = r.lo, end = (int64_t)r.hi + 1, span = end - lo;
        Item* out = items + row_item[i];
        for (int32_t q = 0; q < r.count; ++q) {
            int64_t a, b;
            if (r.step) {
                a = lo + (int64_t)q * r.step;
                b = min(end, a + r.step);
            } else {
                a = lo + span * q / r.count;
                b = lo + span * (q + 1) / r.count;
            }
            out[q] = Item{(int32_t)i, (int32_t)a, (int32_t)b, r.mode};
        }
    }
}

__global__ void k_mode_flags(const Item* __restrict__ items, int64_t nitems, int32_t mode,
                             int32_t* __restrict__ flags) {
    GRID_STRIDE(q, nitems) flags[q] = items[q].mode == mode ? 1 : 0;
}

__global__ void k_mode_list(const int32_t* __restrict__ rank, int64_t nitems,
                            int32_t* __restrict__ list) {
    GRID_STRIDE(q, nitems) {
        const int32_t p = rank[q];
        if (rank[q + 1] != p) list[p] = (int32_t)q;
    }
}

__global__ void k_rowoff(const int32_t* __restrict__ row_item, const int64_t* __restrict__ ioff,
                         int32_t m, int64_t* __restrict__ rowoff) {
    GRID_STRIDE(i, (int64_t)m + 1) rowoff[i] = ioff[row_item[i]];
}

// Window boundaries: row r starts a new window when floor(rowoff[r] / C)
// exceeds floor(rowoff[r-1] / C); with C = cap - (largest row), every window
// then holds at most cap pairs.
__global__ void k_window_flags(const int64_t* __restrict__ rowoff, int32_t m, int64_t C,
                               int32_t* __restrict__ flags) {
    GRID_STRIDE(r, m) flags[r] = (r == 0) ? 1 : ((rowoff[r] / C) != (rowoff[r - 1] / C) ? 1 : 0);
}

__global__ void k_window_list(const int32_t* __restrict__ rank, int32_t m,
                              int32_t* __restrict__ splits) {
    GRID_STRIDE(r, m) {
        const int32_t p = rank[r];
        if (rank[r + 1] != p) splits[p] = (int32_t)r;
    }
}

__global__ void k_max_row(const int64_t* __restrict__ rowoff, int32_t m,
                          unsigned long long* __restrict__ out) {
    unsigned long long best = 0;
    GRID_STRIDE(r, m) {
        const unsigned long long c = (unsigned long long)(rowoff[r + 1] - rowoff[r]);
        best = c > best ? c : best;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, d);
        best = o > best ? o : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(out, best);
}

// Per-handler totals: a row's items all share one mode. Columns (MS_COLS):
// rows, wedges, incidences, pairs, wedges through non-hub vertices, and the
// candidate partners the dense handlers' extraction scans (one hub mask read
// each) in the counting pass and in the fill (which skips items without pairs).
__global__ void k_mode_stats(const int32_t* __restrict__ row_item, const Item* __restrict__ items,
                             const int64_t* __restrict__ W, const int32_t* __restrict__ size,
                             const int64_t* __restrict__ rowoff, const int64_t* __restrict__ ioff,
                             const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                             const int32_t* __restrict__ hubidx, const int32_t* __restrict__ wbeg,
                             const int32_t* __restrict__ wend, const int64_t* __restrict__ Wp,
                             int32_t m, unsigned long long* __restrict__ out) {
    GRID_STRIDE(i, m) {
        const int32_t q0 = row_item[i], q1 = row_item[i + 1];
        if (q1 == q0) continue;
        const int mode = items[q0].mode;
        unsigned long long nonhub = 0, scan_c = 0, scan_f = 0;
        if (mode == MODE_HUBPAIR) {
            nonhub = (unsigned long long)Wp[i];  // entries walked: non-hub wedges + pair hits
        } else {
            for (int32_t e = off[i]; e < off[i + 1]; ++e)
                if (hubidx[idx[e]] < 0) nonhub += (unsigned long long)(wend[e] - wbeg[e]);
        }
        if (mode == MODE_DENSE || mode == MODE_WDENSE) {
            for (int32_t q = q0; q < q1; ++q) {
                const Item it = items[q];
                // the warp handler starts its tiles at a multiple of 32 ids
                const int32_t a = mode == MODE_WDENSE ? (it.jlo & ~31) : it.jlo;
                const unsigned long long n = (unsigned long long)(it.jhi - a);
                scan_c += n;
                if (ioff[q + 1] != ioff[q]) scan_f += n;
            }
        }
        unsigned long long* o = out + mode * MS_COLS;
        atomicAdd(&o[0], 1ull);
        atomicAdd(&o[1], (unsigned long long)W[i]);
        atomicAdd(&o[2], (unsigned long long)size[i]);
        atomicAdd(&o[3], (unsigned long long)(rowoff[i + 1] - rowoff[i]));
        atomicAdd(&o[4], nonhub);
        atomicAdd(&o[5], scan_c);
        atomicAdd(&o[6], scan_f);
    }
}

// Wedges of the rows whose items go to the table or sparse-accumulator handlers.
__global__ void k_sparse_wedges(const int32_t* __restrict__ row_item,
                                const Item* __restrict__ items, const int64_t* __restrict__ W,
                                int32_t m, unsigned long long* __restrict__ out) {
    unsigned long long acc = 0;
    GRID_STRIDE(i, m) {
        const int32_t q = row_item[i];
        if (row_item[i + 1] == q) continue;
        const int mode = items[q].mode;
        if (mode == MODE_BLOCK || mode == MODE_SPARSE || mode == MODE_WSPARSE)
            acc += (unsigned long long)W[i];
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// Entries the sparse-accumulator and hub-pair rows walk (wedges W[i], or the
// hub-pair walk Wp[i]): no row of theirs has more pairs than that.
__global__ void k_stage_bound(const int32_t* __restrict__ row_item, const Item* __restrict__ items,
                              const int64_t* __restrict__ W, const int64_t* __restrict__ Wp,
                              int32_t m, unsigned long long* __restrict__ out) {
    unsigned long long acc = 0;
    GRID_STRIDE(i, m) {
        const int32_t q = row_item[i];
        if (row_item[i + 1] == q) continue;
        const int mode = items[q].mode;
        if (mode == MODE_SPARSE) acc += (unsigned long long)W[i];
        if (mode == MODE_HUBPAIR && Wp) acc += (unsigned long long)max(Wp[i], (int64_t)0);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// rowtot[r] = sum over the k lists of rowoff[t][r] (cumulative, so the sum of
// the lists' row counts before row r)
__global__ void k_sum_rows(const int64_t* __restrict__ rowoff, int32_t k, int32_t m,
                           int64_t* __restrict__ rowtot) {
    GRID_STRIDE(r, (int64_t)m + 1) {
        int64_t acc = 0;
        for (int32_t t = 0; t < k; ++t) acc += rowoff[(int64_t)t * ((int64_t)m + 1) + r];
        rowtot[r] = acc;
    }
}


}  // namespace

void Plan::release_ensemble(cudaStream_t st) {
    dfree(ens.icnt, st);
    dfree(ens.ioff, st);
    dfree(ens.rowoff, st);
    dfree(ens.rowtot, st);
    ens.k = 0;
    ens.counted = false;
}

void Plan::release_stage(cudaStream_t st) {
    dfree(stage_at, st);
    dfree(stage_J, st);
    dfree(stage_O, st);
    dfree(stage_cursor, st);
    stage_cap = 0;
    stage_s = -1;
    stage_bytes_add(-stage_bytes);
    stage_bytes = 0;
}

void Plan::release_stream(cudaStream_t st) {
    dfree(stream_cum, st);
    stream_cum = nullptr;
    stream_k = 0;
}

void Plan::release(cudaStream_t st) {
    release_ensemble(st);
    release_stage(st);
    release_stream(st);
    if (idxTs_owned) dfree(idxTs, st);
    idxTs = nullptr;
    dfree(ks, st);
    dfree(wbeg, st);
    dfree(wend, st);
    dfree(W, st);
    dfree(jmin, st);
    dfree(jmax, st);
    dfree(nnh, st);
    dfree(row_item, st);
    dfree(items, st);
    for (int k = 0; k < NMODES; ++k) {
        dfree(mode_rank[k], st);
        dfree(mode_list[k], st);
        mode_count[k] = 0;
    }
    dfree(icnt, st);
    dfree(ioff, st);
    dfree(rowoff, st);
    if (idxT2s_owned) dfree(idxT2s, st);
    idxT2s = nullptr;
    idxT2s_owned = false;
    dfree(ks2, st);
    dfree(wbeg2, st);
    dfree(wend2, st);
    dfree(Wp, st);
    hp = nullptr;
    s = 0;
    built = false;
    nitems = 0;
    counted = false;
    pairs = wedges = 0;
}

void plan_build(const GraphDev& g, int32_t s, const BinParams& bp, Plan& p, cudaStream_t st,
                const HubPairs* hp) {
    p.release(st);
    p.s = s;
    p.rs = RowS{g.srow, g.rbase, s};
    const int64_t nnz = g.nnz;
    const int32_t m = g.m;
    const int T = 256;

    // pruned transpose
    if (!g.srow && s <= g.min_size) {
        p.idxTs = g.idxT;
        p.idxTs_owned = false;
        p.ks = nullptr;
    } else {
        int32_t* keep = dalloc<int32_t>(nnz, st);
        p.ks = dalloc<int32_t>(nnz + 1, st);
        if (nnz) {
            k_keep_flags<<<grid_for(nnz, T), T, 0, st>>>(g.idxT, g.size, nnz, p.rs, keep);
            SLG_LAUNCH_CHECK();
        }
        scan_i32_to_i32(keep, p.ks, nnz, st);
        dfree(keep, st);
        // +4: the dense handler reads H^T with 16-byte vector loads that may
        // reach up to three entries past the last kept position
        p.idxTs = dalloc<int32_t>(nnz + 4, st);
        SLG_CUDA_TRY(cudaMemsetAsync(p.idxTs, 0, sizeof(int32_t) * (nnz + 4), st));
        p.idxTs_owned = true;
        if (nnz) {
            k_compact<<<grid_for(nnz, T), T, 0, st>>>(g.idxT, p.ks, nnz, p.idxTs);
            SLG_LAUNCH_CHECK();
        }
    }
    p.wbeg = dalloc<int32_t>(nnz, st);
    p.wend = dalloc<int32_t>(nnz, st);
    if (nnz) {
        k_wedge_ranges<<<grid_for(nnz, T), T, 0, st>>>(g.idx, g.rowid, g.size, g.tpos, g.offT, p.ks,
                                                       nnz, p.rs, p.wbeg, p.wend);
        SLG_LAUNCH_CHECK();
    }
    // per-row work
    p.W = dalloc<int64_t>(m, st);
    p.jmin = dalloc<int32_t>(m, st);
    p.jmax = dalloc<int32_t>(m, st);
    p.nnh = dalloc<int32_t>(m, st);
    unsigned long long* wtot = dalloc<unsigned long long>(1, st);
    SLG_CUDA_TRY(cudaMemsetAsync(wtot, 0, sizeof(unsigned long long), st));
    if (m) {
        k_row_work<<<grid_for((int64_t)m * 32, T), T, 0, st>>>(g.off, g.idx, g.hubidx, p.wbeg,
                                                               p.wend, p.idxTs, m, p.W, p.jmin,
                                                               p.jmax, p.nnh, wtot);
        SLG_LAUNCH_CHECK();
    }
    // hub pairs (single graphs at s >= 2): pruned pair lists and per-row work
    int32_t *lo2 = nullptr, *hi2 = nullptr;
    if (hp && hp->built && s >= 2 && !g.srow && m) {
        p.hp = hp;
        const int64_t E2 = hp->E2;
        if (s <= g.min_size) {
            p.idxT2s = hp->idxT2;
            p.idxT2s_owned = false;
            p.ks2 = nullptr;
        } else {
            int32_t* keep = dalloc<int32_t>(E2, st);
            p.ks2 = dalloc<int32_t>(E2 + 1, st);
            k_keep_flags<<<grid_for(E2, T), T, 0, st>>>(hp->idxT2, g.size, E2, p.rs, keep);
            SLG_LAUNCH_CHECK();
            scan_i32_to_i32(keep, p.ks2, E2, st);
            dfree(keep, st);
            p.idxT2s = dalloc<int32_t>(E2 + 4, st);
            SLG_CUDA_TRY(cudaMemsetAsync(p.idxT2s, 0, sizeof(int32_t) * (E2 + 4), st));
            p.idxT2s_owned = true;
            k_compact<<<grid_for(E2, T), T, 0, st>>>(hp->idxT2, p.ks2, E2, p.idxT2s);
            SLG_LAUNCH_CHECK();
        }
        p.wbeg2 = dalloc<int32_t>(E2, st);
        p.wend2 = dalloc<int32_t>(E2, st);
        p.Wp = dalloc<int64_t>(m, st);
        lo2 = dalloc<int32_t>(m, st);
        hi2 = dalloc<int32_t>(m, st);
        k_pair_ranges<<<grid_for((int64_t)m * 32, T), T, 0, st>>>(
            g.off, g.idx, g.size, p.wbeg, p.wend, p.idxTs, hp->hp_id, hp->off2, hp->idx2,
            hp->tpos2, hp->offT2, p.ks2, p.idxT2s, m, p.rs, p.wbeg2, p.wend2, p.Wp, lo2, hi2);
        SLG_LAUNCH_CHECK();
    }
    // items
    int32_t* nitem = dalloc<int32_t>(m, st);
    p.row_item = dalloc<int32_t>((size_t)m + 1, st);
    if (m) {
        k_item_count<<<grid_for(m, T), T, 0, st>>>(p.W, p.jmin, p.jmax, g.size, p.nnh, m, p.rs, bp,
                                                   p.Wp, lo2, hi2, nitem);
        SLG_LAUNCH_CHECK();
    }
    {
        // item ids are int32: refuse a binning that would need more
        int64_t* c64 = dalloc<int64_t>((size_t)m + 1, st);
        scan_i32_to_i64(nitem, c64, m, st);
        int64_t total = 0;
        SLG_CUDA_TRY(cudaMemcpyAsync(&total, c64 + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        SLG_CUDA_TRY(cudaStreamSynchronize(st));
        dfree(c64, st);
        if (total > (int64_t)INT32_MAX - 1) {
            dfree(nitem, st);
            dfree(lo2, st);
            dfree(hi2, st);
            throw Error{SLG_ECAPACITY, "binning needs more than 2^31 work items: raise "
                                       "block_item_wedges or sparse_item_wedges"};
        }
    }
    scan_i32_to_i32(nitem, p.row_item, m, st);
    dfree(nitem, st);
    int32_t nitems32 = 0;
    unsigned long long wtot_h = 0;
    SLG_CUDA_TRY(cudaMemcpyAsync(&nitems32, p.row_item + m, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaMemcpyAsync(&wtot_h, wtot, sizeof(wtot_h), cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(wtot, st);
    p.nitems = nitems32;
    p.wedges = (int64_t)wtot_h;
    p.items = dalloc<Item>(p.nitems, st);
    if (m) {
        k_item_emit<<<grid_for(m, T), T, 0, st>>>(p.W, p.jmin, p.jmax, g.size, p.nnh, m, p.rs, bp,
                                                  p.Wp, lo2, hi2, p.row_item, p.items);
        SLG_LAUNCH_CHECK();
    }
    dfree(lo2, st);
    dfree(hi2, st);
    int32_t* flags = dalloc<int32_t>(p.nitems, st);
    for (int k = 0; k < NMODES; ++k) {
        p.mode_rank[k] = dalloc<int32_t>(p.nitems + 1, st);
        if (p.nitems) {
            k_mode_flags<<<grid_for(p.nitems, T), T, 0, st>>>(p.items, p.nitems, k, flags);
            SLG_LAUNCH_CHECK();
        }
        scan_i32_to_i32(flags, p.mode_rank[k], p.nitems, st);
    }
    dfree(flags, st);
    int32_t counts[NMODES];
    for (int k = 0; k < NMODES; ++k)
        SLG_CUDA_TRY(cudaMemcpyAsync(&counts[k], p.mode_rank[k] + p.nitems, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    for (int k = 0; k < NMODES; ++k) {
        p.mode_count[k] = counts[k];
        p.mode_list[k] = dalloc<int32_t>(counts[k], st);
        if (p.nitems) {
            k_mode_list<<<grid_for(p.nitems, T), T, 0, st>>>(p.mode_rank[k], p.nitems,
                                                             p.mode_list[k]);
            SLG_LAUNCH_CHECK();
        }
    }
    p.icnt = dalloc<int32_t>(p.nitems, st);
    p.ioff = dalloc<int64_t>(p.nitems + 1, st);
    p.rowoff = dalloc<int64_t>((size_t)m + 1, st);
    p.counted = false;
    p.built = true;  // only once complete: a failed build leaves the plan unbuilt
}

void plan_offsets(const GraphDev& g, Plan& p, cudaStream_t st) {
    const int T = 256;
    scan_i32_to_i64(p.icnt, p.ioff, p.nitems, st);
    k_rowoff<<<grid_for((int64_t)g.m + 1, T), T, 0, st>>>(p.row_item, p.ioff, g.m, p.rowoff);
    SLG_LAUNCH_CHECK();
    SLG_CUDA_TRY(cudaMemcpyAsync(&p.pairs, p.ioff + p.nitems, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    p.counted = true;
}

void ensemble_count(const GraphDev& g, Plan& p, const int32_t* s, int32_t k, ModeTimer* mt,
                    cudaStream_t st) {
    p.release_ensemble(st);
    Plan::Ensemble& e = p.ens;
    e.k = k;
    for (int32_t t = 0; t < k; ++t) e.s[t] = s[t];
    const int64_t ni = p.nitems, m1 = (int64_t)g.m + 1;
    e.icnt = dalloc<int32_t>((size_t)(k * ni), st);
    e.ioff = dalloc<int64_t>((size_t)(k * (ni + 1)), st);
    e.rowoff = dalloc<int64_t>((size_t)(k * m1), st);
    e.rowtot = dalloc<int64_t>((size_t)m1, st);
    const int T = 256;
    // the plan's work (pruned at s[0] <= s[t]) with threshold s[t]: a pair
    // with overlap >= s[t] has both sizes >= s[t] >= s[0], so it is there
    run_count_ensemble(g, p, mt, st);
    for (int32_t t = 0; t < k; ++t) {
        scan_i32_to_i64(e.icnt + t * ni, e.ioff + t * (ni + 1), ni, st);
        k_rowoff<<<grid_for(m1, T), T, 0, st>>>(p.row_item, e.ioff + t * (ni + 1), g.m,
                                                e.rowoff + t * m1);
        SLG_LAUNCH_CHECK();
        SLG_CUDA_TRY(cudaMemcpyAsync(&e.pairs[t], e.ioff + t * (ni + 1) + ni, sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, st));
    }
    k_sum_rows<<<grid_for(m1, T), T, 0, st>>>(e.rowoff, k, g.m, e.rowtot);
    SLG_LAUNCH_CHECK();
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    e.counted = true;
}

void plan_mode_stats(const GraphDev& g, const Plan& p, int64_t out[NMODES][MS_COLS],
                     cudaStream_t st, const int64_t* rowoff, const int64_t* ioff) {
    if (!rowoff) rowoff = p.rowoff;
    if (!ioff) ioff = p.ioff;
    unsigned long long* d = dalloc<unsigned long long>(NMODES * MS_COLS, st);
    SLG_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(unsigned long long) * NMODES * MS_COLS, st));
    if (g.m) {
        k_mode_stats<<<grid_for(g.m, 256), 256, 0, st>>>(p.row_item, p.items, p.W, g.size,
                                                         rowoff, ioff, g.off, g.idx,
                                                         g.hubidx, p.wbeg, p.wend, p.Wp, g.m, d);
        SLG_LAUNCH_CHECK();
    }
    unsigned long long h[NMODES * MS_COLS];
    SLG_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(d, st);
    for (int k = 0; k < NMODES; ++k)
        for (int c = 0; c < MS_COLS; ++c) out[k][c] = (int64_t)h[k * MS_COLS + c];
}

int64_t plan_sparse_wedges(const GraphDev& g, const Plan& p, cudaStream_t st) {
    unsigned long long* d = dalloc<unsigned long long>(1, st);
    SLG_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(unsigned long long), st));
    if (g.m) {
        k_sparse_wedges<<<grid_for(g.m, 256), 256, 0, st>>>(p.row_item, p.items, p.W, g.m, d);
        SLG_LAUNCH_CHECK();
    }
    unsigned long long h = 0;
    SLG_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(d, st);
    return (int64_t)h;
}

namespace {
// Entries a walk of rows [r0, r1) reads: wedges through vertices that are not
// mask hubs (a mask hub's share of an overlap is a popcount), and for hub-pair
// rows the entries they walk.
__global__ void k_row_walk(const int32_t* __restrict__ row_item, const Item* __restrict__ items,
                           const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                           const int32_t* __restrict__ hubidx, const int32_t* __restrict__ wbeg,
                           const int32_t* __restrict__ wend, const int64_t* __restrict__ Wp,
                           int32_t r0, int32_t r1, unsigned long long* __restrict__ out) {
    unsigned long long acc = 0;
    for (int64_t r = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < r1;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q0 = row_item[r];
        if (row_item[r + 1] == q0) continue;
        if (items[q0].mode == MODE_HUBPAIR && Wp) {
            acc += (unsigned long long)max(Wp[r], (int64_t)0);
            continue;
        }
        for (int32_t e = off[r]; e < off[r + 1]; ++e)
            if (hubidx[idx[e]] < 0) acc += (unsigned long long)(wend[e] - wbeg[e]);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}
}  // namespace

int64_t plan_row_walk(const GraphDev& g, const Plan& p, int32_t r0, int32_t r1, cudaStream_t st) {
    if (r1 <= r0) return 0;
    unsigned long long* d = dalloc<unsigned long long>(1, st);
    SLG_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(unsigned long long), st));
    k_row_walk<<<grid_for(r1 - r0, 256), 256, 0, st>>>(p.row_item, p.items, g.off, g.idx, g.hubidx,
                                                       p.wbeg, p.wend, p.Wp, r0, r1, d);
    SLG_LAUNCH_CHECK();
    unsigned long long h = 0;
    SLG_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(d, st);
    return (int64_t)h;
}

int64_t plan_stage_bound(const GraphDev& g, const Plan& p, cudaStream_t st) {
    unsigned long long* d = dalloc<unsigned long long>(1, st);
    SLG_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(unsigned long long), st));
    if (g.m) {
        k_stage_bound<<<grid_for(g.m, 256), 256, 0, st>>>(p.row_item, p.items, p.W, p.Wp, g.m, d);
        SLG_LAUNCH_CHECK();
    }
    unsigned long long h = 0;
    SLG_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(d, st);
    return (int64_t)h;
}

namespace {
__global__ void k_count_staged(const int64_t* __restrict__ at, int64_t n,
                               unsigned long long* __restrict__ out) {
    unsigned long long acc = 0;
    GRID_STRIDE(q, n) acc += at[q] >= 0 ? 1ull : 0ull;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}
}  // namespace

int64_t plan_staged_items(const Plan& p, cudaStream_t st) {
    if (!p.stage_at || p.nitems == 0) return 0;
    unsigned long long* d = dalloc<unsigned long long>(1, st);
    SLG_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(unsigned long long), st));
    k_count_staged<<<grid_for(p.nitems, 256), 256, 0, st>>>(p.stage_at, p.nitems, d);
    SLG_LAUNCH_CHECK();
    unsigned long long h = 0;
    SLG_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(d, st);
    return (int64_t)h;
}

int64_t plan_max_row(const GraphDev& g, const int64_t* rowoff, cudaStream_t st) {
    unsigned long long* d = dalloc<unsigned long long>(1, st);
    SLG_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(unsigned long long), st));
    if (g.m) {
        k_max_row<<<grid_for(g.m, 256), 256, 0, st>>>(rowoff, g.m, d);
        SLG_LAUNCH_CHECK();
    }
    unsigned long long h = 0;
    SLG_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(d, st);
    return (int64_t)h;
}

int32_t plan_windows(const GraphDev& g, const int64_t* rowoff, int64_t C, int32_t* splits_dev,
                     cudaStream_t st) {
    const int T = 256;
    const int32_t m = g.m;
    int32_t* flags = dalloc<int32_t>(m, st);
    int32_t* rank = dalloc<int32_t>((size_t)m + 1, st);
    if (m) {
        k_window_flags<<<grid_for(m, T), T, 0, st>>>(rowoff, m, C, flags);
        SLG_LAUNCH_CHECK();
    }
    scan_i32_to_i32(flags, rank, m, st);
    int32_t nw = 0;
    SLG_CUDA_TRY(cudaMemcpyAsync(&nw, rank + m, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    if (splits_dev && m) {
        k_window_list<<<grid_for(m, T), T, 0, st>>>(rank, m, splits_dev);
        SLG_LAUNCH_CHECK();
    }
    dfree(flags, st);
    dfree(rank, st);
    return nw;
}

}  // namespace slg
