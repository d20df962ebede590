// Hub pairs: the counting and fill passes of Algorithm 2 (Section III-C) for
// sparse rows at s >= 2, with the wedges through high-degree vertices replaced
// by an index of hub pairs.
//
// Split the vertices into the K highest-degree ones ("HP hubs") and the rest.
// The overlap of two rows is then |e_i ∩ e_j| = l + t, with l the non-hub
// vertices and t the hubs they share. A pair with overlap >= s >= 2 has l >= 1
// or t >= 2, so its partner j is found either in the wedge range of a non-hub
// vertex of e_i (the ordinary wedges, few, since non-hub vertices have small
// degree) or in the list of rows that hold some pair of e_i's hubs. Rows that
// share t hubs meet in exactly t(t-1)/2 of those pair lists, so per partner
// the handler counts l (non-hub wedges) and c = t(t-1)/2 (pair-list hits) and
// recovers t from c; a partner found through non-hub wedges only (c = 0)
// shares at most one hub, which one look at its hub list settles. Pairs that
// share just one hub and nothing else (overlap 1 < s) are never enumerated:
// on hub-heavy inputs those are most of Algorithm 2's wedges.
//
// One CTA per work item (row i, partners in [jlo, jhi)): the item's slices of
// all its ranges are loaded as one flat list into a shared-memory
// open-addressing table (16-bit non-hub count, 16-bit pair count per
// partner); a slice with more distinct partners than the table may hold is
// redone as two halves. Survivors are sorted by j and written in order.
#include <algorithm>
#include <vector>

#include "kernel_util.cuh"
#include "plan.cuh"

namespace slg {
namespace {

#define GRID_STRIDE(k, n)                                                            \
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < (n);       \
         k += (int64_t)gridDim.x * blockDim.x)

int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

// ---------------------------------------------------------------- build

constexpr int HB_BINS = 1 << 20;  // degree histogram (higher degrees share the last bin)

__global__ void k_deg_hist(const int32_t* __restrict__ offT, int32_t n, int32_t* __restrict__ hist) {
    GRID_STRIDE(v, n) {
        const int32_t d = offT[v + 1] - offT[v];
        if (d >= 2) atomicAdd(&hist[min(d, HB_BINS - 1)], 1);
    }
}

// Per row: k_i = its vertices of degree >= dmin; total += C(k_i, 2).
__global__ void k_row_hubs(const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                           const int32_t* __restrict__ offT, int32_t dmin, int32_t m,
                           int32_t* __restrict__ k_out, unsigned long long* __restrict__ total) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long acc = 0;
    for (int64_t i = warp; i < m; i += nwarps) {
        int32_t k = 0;
        for (int32_t e = off[i] + lane; e < off[i + 1]; e += 32) {
            const int32_t v = idx[e];
            k += (offT[v + 1] - offT[v] >= dmin) ? 1 : 0;
        }
        k = (int32_t)__reduce_add_sync(0xffffffffu, (unsigned)k);
        if (lane == 0) {
            if (k_out) k_out[i] = k;
            acc += (unsigned long long)k * (unsigned long long)(k - 1) / 2ull;
        }
    }
    if (lane == 0 && acc) atomicAdd(total, acc);
}

__global__ void k_hub_flags(const int32_t* __restrict__ offT, int32_t n, int32_t dmin,
                            int32_t* __restrict__ flags) {
    GRID_STRIDE(v, n) flags[v] = (offT[v + 1] - offT[v] >= dmin) ? 1 : 0;
}

__global__ void k_hub_number(const int32_t* __restrict__ rank, int32_t n,
                             int32_t* __restrict__ hp_id) {
    GRID_STRIDE(v, n) hp_id[v] = rank[v + 1] != rank[v] ? rank[v] : -1;
}

// Row i's hub numbers, in vertex order (hence ascending), at hlist[hoff[i]..].
__global__ void k_row_hublist(const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                              const int32_t* __restrict__ hp_id, const int32_t* __restrict__ hoff,
                              int32_t m, int32_t* __restrict__ hlist) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < m; i += nwarps) {
        int32_t at = hoff[i];
        for (int32_t eb = off[i]; eb < off[i + 1]; eb += 32) {
            const int32_t e = eb + lane;
            const int32_t h = e < off[i + 1] ? hp_id[idx[e]] : -1;
            const unsigned bal = __ballot_sync(0xffffffffu, h >= 0);
            if (h >= 0) hlist[at + __popc(bal & lt)] = h;
            at += __popc(bal);
        }
    }
}

__global__ void k_big_flags(const int32_t* __restrict__ hoff, int32_t m, int32_t bigk,
                            int32_t* __restrict__ flags) {
    GRID_STRIDE(i, m) flags[i] = (hoff[i + 1] - hoff[i] > bigk) ? 1 : 0;
}

__global__ void k_big_number(const int32_t* __restrict__ rank, int32_t m,
                             int32_t* __restrict__ bigidx) {
    GRID_STRIDE(i, m) bigidx[i] = rank[i + 1] != rank[i] ? rank[i] : -1;
}

// Hub bitmap of each row that has one (one warp per row).
__global__ void k_big_bits(const int32_t* __restrict__ hoff, const int32_t* __restrict__ hlist,
                           const int32_t* __restrict__ bigidx, int32_t m,
                           uint32_t* __restrict__ bigbits) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < m; i += nwarps) {
        const int32_t b = bigidx[i];
        if (b < 0) continue;
        uint32_t* bits = bigbits + (int64_t)b * (HP_MAXK / 32);
        for (int32_t x = hoff[i] + lane; x < hoff[i + 1]; x += 32) {
            const int32_t h = hlist[x];
            atomicOr(&bits[h >> 5], 1u << (h & 31));
        }
    }
}

// Row i's look record (a thread per row).
__global__ void k_row_records(const int32_t* __restrict__ hoff, const int32_t* __restrict__ hlist,
                              int32_t m, uint4* __restrict__ hrec) {
    GRID_STRIDE(i, m) {
        const int32_t h0 = hoff[i], nh = hoff[i + 1] - h0;
        uint32_t w[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) w[k] = 0u;
        if (nh > 31) {
            w[0] = 0xffffu;
        } else {
            w[0] = (uint32_t)nh;
            for (int32_t k = 0; k < nh; ++k) {
                const int32_t pos = k + 1;
                const uint32_t id = (uint32_t)hlist[h0 + k];
#pragma unroll
                for (int x = 0; x < 16; ++x)
                    if (x == (pos >> 1)) w[x] |= id << ((pos & 1) * 16);
            }
        }
        uint4* r = hrec + (int64_t)i * 4;
        r[0] = make_uint4(w[0], w[1], w[2], w[3]);
        r[1] = make_uint4(w[4], w[5], w[6], w[7]);
        r[2] = make_uint4(w[8], w[9], w[10], w[11]);
        r[3] = make_uint4(w[12], w[13], w[14], w[15]);
    }
}

__global__ void k_pair_counts(const int32_t* __restrict__ hoff, int32_t m,
                              int32_t* __restrict__ np) {
    GRID_STRIDE(i, m) {
        const int64_t k = hoff[i + 1] - hoff[i];
        np[i] = (int32_t)(k * (k - 1) / 2);
    }
}

// Row i's pair keys a*K + b (a < b its hub numbers), ascending, and their row.
__global__ void k_row_pairs(const int32_t* __restrict__ hoff, const int32_t* __restrict__ hlist,
                            const int32_t* __restrict__ off2, int32_t m, int32_t K,
                            int32_t* __restrict__ idx2, int32_t* __restrict__ rowid2) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < m; i += nwarps) {
        const int32_t h0 = hoff[i];
        const int64_t k = hoff[i + 1] - h0;
        const int64_t base = off2[i];
        for (int64_t a = 0; a + 1 < k; ++a) {
            const int64_t first = base + a * (2 * k - a - 1) / 2;  // pairs (a, a+1..k-1)
            const int32_t ha = hlist[h0 + a];
            for (int64_t b = a + 1 + lane; b < k; b += 32) {
                const int64_t pos = first + (b - a - 1);
                idx2[pos] = ha * K + hlist[h0 + b];
                rowid2[pos] = (int32_t)i;
            }
        }
    }
}

}  // namespace

void HubPairs::release(cudaStream_t st) {
    dfree(hp_id, st);
    dfree(hoff, st);
    dfree(hlist, st);
    dfree(off2, st);
    dfree(idx2, st);
    dfree(offT2, st);
    dfree(idxT2, st);
    dfree(tpos2, st);
    dfree(bigidx, st);
    dfree(bigbits, st);
    dfree(hrec, st);
    bigk = 0;
    built = false;
    K = 0;
    E1 = E2 = 0;
}

void hubpair_build(const GraphDev& g, int32_t max_hubs, int64_t max_pairs, HubPairs& hp,
                   cudaStream_t st) {
    hp.release(st);
    hp.tried = true;
    const int32_t m = g.m, n = g.n;
    if (m == 0 || n == 0 || max_hubs < 2) return;
    // memory: the pair incidences, their rows, the transpose's outputs and its
    // four scratch arrays take about 32 bytes per hub-pair incidence
    size_t free_b = 0, total_b = 0;
    SLG_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    const int64_t by_mem = (int64_t)((free_b > ((size_t)4 << 30) ? free_b - ((size_t)4 << 30) : 0) / 40);
    max_pairs = std::min<int64_t>(std::min<int64_t>(max_pairs, by_mem), (int64_t)INT32_MAX - 64);
    // degree threshold for at most max_hubs hubs
    int32_t* hist = dalloc<int32_t>(HB_BINS, st);
    SLG_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(int32_t) * HB_BINS, st));
    k_deg_hist<<<grid_for(n, 256), 256, 0, st>>>(g.offT, n, hist);
    SLG_LAUNCH_CHECK();
    std::vector<int32_t> hh(HB_BINS);
    SLG_CUDA_TRY(cudaMemcpyAsync(hh.data(), hist, sizeof(int32_t) * HB_BINS, cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(hist, st);
    std::vector<int64_t> atleast(HB_BINS + 1, 0);  // vertices with degree >= d (d >= 2)
    for (int32_t d = HB_BINS - 1; d >= 0; --d) atleast[d] = atleast[d + 1] + hh[d];
    auto threshold_for = [&](int64_t count) {  // smallest d >= 2 with atleast[d] <= count
        int32_t d = 2;
        while (d < HB_BINS && atleast[d] > count) ++d;
        return d;
    };
    int64_t want = max_hubs;
    int32_t dmin = threshold_for(want);
    unsigned long long* tot = dalloc<unsigned long long>(1, st);
    int64_t E2 = 0;
    for (int guard = 0; guard < 40; ++guard) {
        if (dmin >= HB_BINS - 1 || atleast[dmin] < 2) break;
        SLG_CUDA_TRY(cudaMemsetAsync(tot, 0, sizeof(unsigned long long), st));
        k_row_hubs<<<grid_for((int64_t)m * 32, 256), 256, 0, st>>>(g.off, g.idx, g.offT, dmin, m,
                                                                    nullptr, tot);
        SLG_LAUNCH_CHECK();
        unsigned long long t = 0;
        SLG_CUDA_TRY(cudaMemcpyAsync(&t, tot, sizeof(t), cudaMemcpyDeviceToHost, st));
        SLG_CUDA_TRY(cudaStreamSynchronize(st));
        E2 = (int64_t)t;
        if (E2 <= max_pairs) break;
        want = atleast[dmin] / 2;  // halve the hubs
        dmin = threshold_for(want);
        E2 = 0;
    }
    if (dmin >= HB_BINS - 1 || atleast[dmin] < 2 || E2 == 0 || E2 > max_pairs) {
        dfree(tot, st);
        return;
    }
    const int32_t K = (int32_t)atleast[dmin];
    // hub numbers in vertex order
    int32_t* flags = dalloc<int32_t>(n, st);
    int32_t* rank = dalloc<int32_t>((size_t)n + 1, st);
    k_hub_flags<<<grid_for(n, 256), 256, 0, st>>>(g.offT, n, dmin, flags);
    SLG_LAUNCH_CHECK();
    scan_i32_to_i32(flags, rank, n, st);
    hp.hp_id = dalloc<int32_t>(n, st);
    k_hub_number<<<grid_for(n, 256), 256, 0, st>>>(rank, n, hp.hp_id);
    SLG_LAUNCH_CHECK();
    dfree(flags, st);
    dfree(rank, st);
    // row hub lists
    int32_t* kr = dalloc<int32_t>(m, st);
    SLG_CUDA_TRY(cudaMemsetAsync(tot, 0, sizeof(unsigned long long), st));
    k_row_hubs<<<grid_for((int64_t)m * 32, 256), 256, 0, st>>>(g.off, g.idx, g.offT, dmin, m, kr, tot);
    SLG_LAUNCH_CHECK();
    hp.hoff = dalloc<int32_t>((size_t)m + 1, st);
    scan_i32_to_i32(kr, hp.hoff, m, st);
    int32_t E1 = 0;
    SLG_CUDA_TRY(cudaMemcpyAsync(&E1, hp.hoff + m, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    hp.E1 = E1;
    hp.hlist = dalloc<int32_t>((size_t)E1 + 1, st);
    k_row_hublist<<<grid_for((int64_t)m * 32, 256), 256, 0, st>>>(g.off, g.idx, hp.hp_id, hp.hoff,
                                                                   m, hp.hlist);
    SLG_LAUNCH_CHECK();
    // hub bitmaps of the rows with many hubs (at most 2^22 rows: 2 GiB)
    {
        int32_t* flags = dalloc<int32_t>(m, st);
        int32_t* rank = dalloc<int32_t>((size_t)m + 1, st);
        int32_t bigk = 32, nbig = 0;
        for (;; bigk *= 2) {
            k_big_flags<<<grid_for(m, 256), 256, 0, st>>>(hp.hoff, m, bigk, flags);
            SLG_LAUNCH_CHECK();
            scan_i32_to_i32(flags, rank, m, st);
            SLG_CUDA_TRY(cudaMemcpyAsync(&nbig, rank + m, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            SLG_CUDA_TRY(cudaStreamSynchronize(st));
            if (nbig <= (1 << 22)) break;
        }
        hp.bigk = bigk;
        hp.bigidx = dalloc<int32_t>(m, st);
        k_big_number<<<grid_for(m, 256), 256, 0, st>>>(rank, m, hp.bigidx);
        SLG_LAUNCH_CHECK();
        const size_t words = (size_t)(nbig > 0 ? nbig : 1) * (HP_MAXK / 32);
        hp.bigbits = dalloc<uint32_t>(words, st);
        SLG_CUDA_TRY(cudaMemsetAsync(hp.bigbits, 0, sizeof(uint32_t) * words, st));
        if (nbig > 0) {
            k_big_bits<<<grid_for((int64_t)m * 32, 256), 256, 0, st>>>(hp.hoff, hp.hlist, hp.bigidx,
                                                                        m, hp.bigbits);
            SLG_LAUNCH_CHECK();
        }
        dfree(flags, st);
        dfree(rank, st);
    }
    hp.hrec = dalloc<uint4>((size_t)m * 4, st);
    k_row_records<<<grid_for(m, 256), 256, 0, st>>>(hp.hoff, hp.hlist, m, hp.hrec);
    SLG_LAUNCH_CHECK();
    // hub-pair incidences and their transpose
    k_pair_counts<<<grid_for(m, 256), 256, 0, st>>>(hp.hoff, m, kr);
    SLG_LAUNCH_CHECK();
    hp.off2 = dalloc<int32_t>((size_t)m + 1, st);
    scan_i32_to_i32(kr, hp.off2, m, st);
    dfree(kr, st);
    dfree(tot, st);
    hp.E2 = E2;
    hp.K = K;
    hp.idx2 = dalloc<int32_t>((size_t)E2, st);
    int32_t* rowid2 = dalloc<int32_t>((size_t)E2, st);
    k_row_pairs<<<grid_for((int64_t)m * 32, 256), 256, 0, st>>>(hp.hoff, hp.hlist, hp.off2, m, K,
                                                                hp.idx2, rowid2);
    SLG_LAUNCH_CHECK();
    const int32_t n2 = K * K;
    hp.offT2 = dalloc<int32_t>((size_t)n2 + 1, st);
    hp.idxT2 = dalloc<int32_t>((size_t)E2 + 4, st);
    hp.tpos2 = dalloc<int32_t>((size_t)E2, st);
    build_transpose(hp.idx2, rowid2, n2, E2, hp.offT2, hp.idxT2, hp.tpos2, st);
    dfree(rowid2, st);
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    hp.built = true;
}

namespace {

// ---------------------------------------------------------------- kernel

constexpr int HP_THREADS = 512;
constexpr int HP_TABLE = 6144;           // slots (key + packed counts): 48 KB, three CTAs per SM
constexpr int HP_CAP = HP_TABLE / 2;     // distinct partners before a slice splits
constexpr int HP_WORDS = HP_MAXK / 32;   // hub bitmap of the row
constexpr int HP_SLOTS_PER_THREAD = HP_TABLE / HP_THREADS;
constexpr int HP_RANGES = (SP_MAX_SIZE + HP_MAXR + 31) & ~31;  // ranges of a row, at most
// per-CTA scratch in device memory: range cursors, and the fill's survivors
constexpr int HP_SCRATCH_WORDS = 2 * HP_RANGES + 2 * HP_CAP;
constexpr uint32_t HP_LIGHT = 0x10000u;  // a non-hub wedge (high half); a pair-list hit adds 1
constexpr int32_t HP_EMPTY = -1;
constexpr int HP_BUCKETS = 1024;         // fill: survivors are bucketed by j before sorting
static_assert(HP_TABLE % HP_THREADS == 0 && HP_ITEM <= HP_CAP, "table and item sizes");
static_assert(HP_CAP <= 65535, "look list holds 16-bit slots");
static_assert(HP_BUCKETS % HP_THREADS == 0 && 2 * (HP_BUCKETS + 1) <= HP_CAP + 32,
              "bucket counts fit the look list's storage");
constexpr size_t HP_SMEM = sizeof(int32_t) * HP_TABLE * 2;

__device__ __forceinline__ uint32_t hp_slot(int32_t j) {
    return (uint32_t)(((uint64_t)((uint32_t)j * 2654435761u) * HP_TABLE) >> 32);
}

// Insert-or-add (linear probing); keys go EMPTY -> j once. Returns 1 when the
// key was created, 0 when it existed, -1 when no slot was free.
__device__ __forceinline__ int hp_add(int32_t* keys, uint32_t* cnts, int32_t j, uint32_t inc) {
    uint32_t h = hp_slot(j);
    volatile int32_t* vk = keys;
    for (int probe = 0; probe < HP_TABLE; ++probe) {
        const int32_t k = vk[h];
        if (k == j) {
            atomicAdd(&cnts[h], inc);
            return 0;
        }
        if (k == HP_EMPTY) {
            const int32_t old = atomicCAS(&keys[h], HP_EMPTY, j);
            if (old == HP_EMPTY || old == j) {
                atomicAdd(&cnts[h], inc);
                return old == HP_EMPTY ? 1 : 0;
            }
        }
        h = h + 1 == HP_TABLE ? 0 : h + 1;
    }
    return -1;
}

// t from c = t(t-1)/2, exactly (c < 2^16).
__device__ __forceinline__ int32_t hubs_from_pairs(uint32_t c) {
    const uint32_t x = 1u + 8u * c;  // (2t - 1)^2
    uint32_t r = (uint32_t)sqrtf((float)x);
    while (r * r > x) --r;
    while ((r + 1) * (r + 1) <= x) ++r;
    return (int32_t)((r + 1) >> 1);
}

// First position in [c, t) whose entry is >= b (src ascending there): the
// last entry first, then galloping from c (a slice usually holds few entries
// of a range), then a binary search of the last step.
__device__ __forceinline__ int32_t gallop_to(const int32_t* __restrict__ src, int32_t c,
                                             int32_t t, int32_t b) {
    if (c >= t || __ldg(&src[t - 1]) < b) return t;
    if (__ldg(&src[c]) >= b) return c;
    int32_t lo = c, step = 1, hi = t;  // src[lo] < b
    for (;;) {
        const int32_t p = lo + step;
        if (p >= t - 1) break;  // src[t - 1] >= b
        if (__ldg(&src[p]) >= b) {
            hi = p;
            break;
        }
        lo = p;
        step <<= 1;
    }
    return lower_bound_dev(src, lo + 1, hi, b);
}

// One CTA takes a row (it claims the row's first item and walks all of the
// row's items in this launch in order, so each range keeps a cursor at the
// first entry of the next slice and only the slice's end is searched).
// ENS4: the counting pass of an ensemble of at most four lists (*eap, in device
// memory): every list counted in the one walk.
template <bool FILL, bool ENS4 = false>
__global__ void __launch_bounds__(HP_THREADS, 3)
k_hubpair_items(const Item* __restrict__ items, const int32_t* __restrict__ list,
                const int32_t* __restrict__ rank, int32_t item_lo, int32_t item_hi,
                const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                const int32_t* __restrict__ wbeg, const int32_t* __restrict__ wend,
                const int32_t* __restrict__ idxTs, const int32_t* __restrict__ hp_id,
                const int32_t* __restrict__ hoff, const int32_t* __restrict__ hlist,
                const int32_t* __restrict__ bigidx, const uint32_t* __restrict__ bigbits,
                const uint4* __restrict__ hrec, int32_t bigk, const int32_t* __restrict__ off2, const int32_t* __restrict__ wbeg2,
                const int32_t* __restrict__ wend2, const int32_t* __restrict__ idxT2s, RowS rs,
                int32_t* __restrict__ icnt, const int64_t* __restrict__ ioff,
                int32_t* __restrict__ I, int32_t* __restrict__ J, int32_t* __restrict__ O,
                int32_t* __restrict__ queue, int64_t limit, int32_t* __restrict__ err,
                int32_t* __restrict__ scratch, StageArgs sa, const EnsArgs* __restrict__ eap) {
    static_assert(!(FILL && ENS4), "an ensemble's lists are counted here, filled one at a time");
    constexpr int NT = HP_THREADS;
    const bool stg = FILL && sa.J != nullptr;  // the counting pass, staging pairs
    int32_t* cur = scratch + (int64_t)blockIdx.x * HP_SCRATCH_WORDS;  // first entry of the next slice
    int32_t* nxt = cur + HP_RANGES;                                   // first entry after this slice
    unsigned long long* surv = reinterpret_cast<unsigned long long*>(nxt + HP_RANGES);  // fill
    extern __shared__ __align__(16) int32_t hp_dyn[];
    int32_t* keys = hp_dyn;                                              // HP_TABLE
    uint32_t* cnts = reinterpret_cast<uint32_t*>(hp_dyn + HP_TABLE);     // HP_TABLE
    unsigned long long* sortbuf = reinterpret_cast<unsigned long long*>(hp_dyn);  // fill
    __shared__ uint32_t hbits[HP_WORDS];
    __shared__ int32_t hmine[SP_MAX_SIZE + 1];  // the row's hubs (|e_i| <= 255)
    __shared__ int32_t pre[NT + 1];
    __shared__ int32_t sub[NT];
    __shared__ int32_t stk_a[64], stk_b[64];
    __shared__ int32_t tmp[NT / 32 + 1];
    __shared__ int32_t sh_pos, sh_n, sh_a, sh_b, sh_nchk;
    __shared__ volatile int32_t nkeys, ovf;
    __shared__ __align__(16) uint16_t chk[HP_CAP + 32];  // slots needing a look; fill: buckets
    __shared__ long long sh_cpos, sh_cend;  // staging: the CTA's chunk of the pool
    __shared__ int32_t sh_sovf, sh_dry;     // staging: the item did not fit; the pool is spent
    const int tid = threadIdx.x;
    const int32_t lo_r = rank[item_lo], hi_r = rank[item_hi];
    for (int t = tid; t < HP_TABLE; t += NT) {
        keys[t] = HP_EMPTY;
        cnts[t] = 0u;
    }
    bool clean = true;  // the table is empty (same in every thread)
    if (tid == 0) {
        sh_cpos = sh_cend = 0;
        sh_dry = 0;
    }
    // a fill item needs its pass: it has pairs and was not staged
    auto needs_fill = [&](int32_t qn) {
        return ioff[qn + 1] != ioff[qn] && !(sa.at && sa.at[qn] >= 0);
    };

    for (;;) {
        // a spent pool ends the staging launch; the counting kernel takes the
        // rows from this queue position on
        if (tid == 0) sh_pos = sh_dry ? hi_r : lo_r + atomicAdd(queue, 1);
        __syncthreads();
        const int32_t pos = sh_pos;
        if (pos >= hi_r) break;
        const int32_t q = list[pos];
        const int32_t i = items[q].row;
        // a row belongs to the CTA that claims its first item
        if (pos > lo_r && items[list[pos - 1]].row == i) {
            __syncthreads();  // everyone has read sh_pos before thread 0 rewrites it
            continue;
        }
        if (FILL && !stg) {
            // a row with nothing left to write (no pairs, or staged) is passed over
            bool want = false;
            for (int32_t k = pos + tid; k < hi_r; k += NT) {
                const int32_t qk = list[k];
                if (items[qk].row != i) break;
                if (needs_fill(qk)) {
                    want = true;
                    break;
                }
            }
            if (!__syncthreads_or(want)) continue;
        }
        const int32_t s = rs.s_of(i);
        const int32_t ib = rs.base_of(i);
        const int32_t e0 = off[i], ne = min(off[i + 1] - e0, SP_MAX_SIZE);
        const int32_t f0 = off2[i], nf = min(off2[i + 1] - f0, HP_MAXR);
        const int32_t nr = ne + nf;
        // the row's hubs, and each range's cursor at its start (every entry lies
        // at or after the row's first item)
        for (int w = tid; w < HP_WORDS; w += NT) hbits[w] = 0u;
        __syncthreads();
        const int32_t ki = min(hoff[i + 1] - hoff[i], SP_MAX_SIZE);
        for (int32_t x = tid; x < ki; x += NT) {
            const int32_t hh = hlist[hoff[i] + x];
            hmine[x] = hh;
            atomicOr(&hbits[hh >> 5], 1u << (hh & 31));
        }
        for (int32_t r = tid; r < nr; r += NT) cur[r] = r < ne ? wbeg[e0 + r] : wbeg2[f0 + r - ne];
        __syncthreads();
        for (int32_t pp = pos; pp < hi_r; ++pp) {
            int32_t qq = pp == pos ? q : list[pp];
            Item it = items[qq];
            if (it.row != i) break;
            bool skip = false;  // cursors only: move them to the next item to fill
            if (FILL && !stg && !needs_fill(qq)) {
                int32_t pn = pp + 1;
                while (pn < hi_r) {
                    const int32_t qn = list[pn];
                    if (items[qn].row != i) {
                        pn = hi_r;
                        break;
                    }
                    if (needs_fill(qn)) break;
                    ++pn;
                }
                if (pn >= hi_r) break;  // no item of the row left with pairs
                it.jhi = items[list[pn]].jlo;
                pp = pn - 1;
                skip = true;
            }
            if (stg) {
                if (tid == 0) {
                    sh_sovf = 0;
                    if (sh_cend - sh_cpos < sa.min_room && !sh_dry) {  // a fresh chunk, if any
                        const unsigned long long c =
                            atomicAdd(sa.cursor, (unsigned long long)sa.chunk);
                        if ((int64_t)c + sa.chunk <= sa.cap) {
                            sh_cpos = (long long)c;
                            sh_cend = (long long)c + sa.chunk;
                        } else {
                            sh_dry = 1;  // the row's items left are counted, not staged
                        }
                    }
                    if (sh_dry) sh_cend = sh_cpos;
                }
                __syncthreads();
            }
            const int64_t obase = !FILL ? 0 : stg ? (int64_t)sh_cpos : ioff[qq] - ioff[item_lo];
            const int64_t olimit = stg ? (int64_t)sh_cend : limit;
            int64_t out_pos = 0;  // same value in every thread
            // ENS4: this thread's survivors of each list in the item so far, and
            // the thresholds (a list beyond the ensemble never counts)
            int32_t en0 = 0, en1 = 0, en2 = 0, en3 = 0;
            const uint32_t es0 = ENS4 ? (uint32_t)eap->s[0] : 0u;
            const uint32_t es1 = ENS4 && eap->k > 1 ? (uint32_t)eap->s[1] : 0xffffffffu;
            const uint32_t es2 = ENS4 && eap->k > 2 ? (uint32_t)eap->s[2] : 0xffffffffu;
            const uint32_t es3 = ENS4 && eap->k > 3 ? (uint32_t)eap->s[3] : 0xffffffffu;
            if (tid == 0) {
                sh_n = 1;
                stk_a[0] = it.jlo;
                stk_b[0] = it.jhi;
            }
            for (;;) {
                __syncthreads();
                const int32_t n_now = sh_n;
                __syncthreads();  // every thread has read sh_n before thread 0 pops
                if (n_now == 0) break;
                if (tid == 0) {
                    sh_n = n_now - 1;
                    sh_a = stk_a[n_now - 1];
                    sh_b = stk_b[n_now - 1];
                    nkeys = 0;
                    ovf = 0;
                }
                if (!clean && !skip) {
                    for (int t = tid; t < HP_TABLE; t += NT) {
                        keys[t] = HP_EMPTY;
                        cnts[t] = 0u;
                    }
                    clean = true;
                }
                __syncthreads();
                const int32_t b = sh_b;
                // each range's slice [cur, nxt): its entries below b
                for (int32_t r = tid; r < nr; r += NT) {
                    int32_t t;
                    const int32_t* src;
                    if (r < ne) {
                        const int32_t e = e0 + r;
                        t = hp_id[idx[e]] < 0 ? wend[e] : cur[r];  // hubs: via the pair lists
                        src = idxTs;
                    } else {
                        t = wend2[f0 + r - ne];
                        src = idxT2s;
                    }
                    nxt[r] = gallop_to(src, cur[r], t, b);
                }
                __syncthreads();
                if (skip) {
                    for (int32_t r = tid; r < nr; r += NT) cur[r] = nxt[r];
                    continue;  // the item has no pair: only the cursors move
                }
                // the slices as one flat list per pass: non-hub wedges (idxTs),
                // then hub-pair hits (idxT2s)
                for (int pass = 0; pass < 2 && !ovf; ++pass) {
                    const int32_t r0 = pass == 0 ? 0 : ne, r1 = pass == 0 ? ne : nr;
                    const int32_t* src = pass == 0 ? idxTs : idxT2s;
                    const uint32_t inc = pass == 0 ? HP_LIGHT : 1u;
                    for (int32_t rb = r0; rb < r1; rb += NT) {
                        const int32_t r = rb + tid;
                        int32_t lo = 0, len = 0;
                        if (r < r1) {
                            lo = cur[r];
                            len = nxt[r] - lo;
                        }
                        int32_t total;
                        const int32_t ex = block_excl_scan<NT>(len, &total, tmp);
                        pre[tid] = ex;
                        sub[tid] = lo;
                        if (tid == 0) pre[NT] = total;
                        __syncthreads();
                        // whole warps walk the flat list together (new keys are
                        // counted once per warp and step)
                        const int32_t tend = (total + 31) & ~31;
                        for (int32_t t = tid; t < tend; t += NT) {
                            // another warp may set the flag at any time: the warp
                            // decides together, so the ballots below see every lane
                            if (__any_sync(0xffffffffu, ovf != 0)) break;
                            int rr = 0;
                            if (t < total) {
                                int32_t x = 0, z = NT - 1;  // largest x with pre[x] <= t
                                while (x < z) {
                                    const int32_t mid = (x + z + 1) >> 1;
                                    if (pre[mid] <= t)
                                        x = mid;
                                    else
                                        z = mid - 1;
                                }
                                rr = hp_add(keys, cnts, __ldg(&src[sub[x] + t - pre[x]]), inc);
                            }
                            const unsigned created = __ballot_sync(0xffffffffu, rr > 0);
                            const unsigned full = __ballot_sync(0xffffffffu, rr < 0);
                            if ((tid & 31) == 0) {
                                if (full || (created &&
                                             atomicAdd((int32_t*)&nkeys, __popc(created)) +
                                                     __popc(created) > HP_CAP))
                                    ovf = 1;
                            }
                        }
                        clean = false;
                        __syncthreads();
                        if (ovf) break;
                    }
                }
                if (ovf) {
                    // more distinct partners than the table may hold: two halves,
                    // the lower first (the cursors have not moved)
                    if (tid == 0) {
                        const int32_t a = sh_a;
                        const int32_t mid = a + (b - a) / 2;
                        stk_a[sh_n] = mid;
                        stk_b[sh_n] = b;
                        stk_a[sh_n + 1] = a;
                        stk_b[sh_n + 1] = mid;
                        sh_n += 2;
                    }
                    __syncthreads();
                    continue;
                }
                for (int32_t r = tid; r < nr; r += NT) cur[r] = nxt[r];
                // survivors: overlap = non-hub count + shared hubs. A pair hit
                // gives the hubs from the pair count; a partner without one shares
                // at most one hub, settled by a look at its hubs. The slots that
                // need a look are listed first, then the whole CTA takes the looks.
                // Each slot's count becomes its overlap if it survives, else 0.
                if (tid == 0) sh_nchk = 0;
                __syncthreads();
#pragma unroll
                for (int r = 0; r < HP_SLOTS_PER_THREAD; ++r) {
                    const int slot = r * NT + tid;
                    const int32_t j = keys[slot];
                    uint32_t outv = 0u;
                    bool needs = false;
                    if (j != HP_EMPTY) {
                        const uint32_t c = cnts[slot];
                        const int32_t l = (int32_t)(c >> 16), pc = (int32_t)(c & 0xffffu);
                        if (pc > 0) {
                            const int32_t ov = l + hubs_from_pairs((uint32_t)pc);
                            outv = ov >= s ? (uint32_t)ov : 0u;
                        } else if (l + 1 >= s) {
                            outv = (uint32_t)l;  // + the shared hub, if any
                            needs = true;
                        }
                    }
                    cnts[slot] = outv;
                    const unsigned bal = __ballot_sync(0xffffffffu, needs);
                    int32_t at = 0;
                    if ((tid & 31) == 0 && bal) at = atomicAdd(&sh_nchk, __popc(bal));
                    at = __shfl_sync(0xffffffffu, at, 0);
                    if (needs) chk[at + __popc(bal & ((1u << (tid & 31)) - 1u))] = (uint16_t)slot;
                }
                __syncthreads();
                const int32_t nchk = sh_nchk;
                // two looks in flight per thread: the partner's record (its hub
                // count and first 15 hubs in one 32-byte sector, 16 more in the
                // next) against the row's bitmap
                for (int32_t xb = tid; xb < nchk; xb += 2 * NT) {
                    int slotv[2];
                    int32_t jv[2], nh[2], tv[2];
                    uint4 ra[2], rb[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int32_t x = xb + u * NT;
                        slotv[u] = x < nchk ? (int)chk[x] : -1;
                        jv[u] = slotv[u] >= 0 ? keys[slotv[u]] : 0;
                        ra[u] = rb[u] = make_uint4(0u, 0u, 0u, 0u);
                        if (slotv[u] >= 0) {
                            ra[u] = __ldg(&hrec[(int64_t)jv[u] * 4]);
                            rb[u] = __ldg(&hrec[(int64_t)jv[u] * 4 + 1]);
                        }
                    }
                    // hub k of a record (1 <= k <= 31) is 16-bit field k
                    auto hit = [&](uint32_t word, int half) {
                        const uint32_t id = (word >> (half * 16)) & 0xffffu;
                        return ((hbits[id >> 5] >> (id & 31)) & 1u) != 0u;
                    };
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        nh[u] = (int32_t)(ra[u].x & 0xffffu);
                        tv[u] = 0;
                        if (slotv[u] < 0 || nh[u] > 31) continue;
                        const uint32_t f[8] = {ra[u].x, ra[u].y, ra[u].z, ra[u].w,
                                               rb[u].x, rb[u].y, rb[u].z, rb[u].w};
#pragma unroll
                        for (int k = 1; k < 16; ++k)
                            if (k <= nh[u] && hit(f[k >> 1], k & 1)) tv[u] = 1;
                        if (nh[u] > 15 && !tv[u]) {
                            const uint4 c = __ldg(&hrec[(int64_t)jv[u] * 4 + 2]);
                            const uint4 d = __ldg(&hrec[(int64_t)jv[u] * 4 + 3]);
                            const uint32_t g2[8] = {c.x, c.y, c.z, c.w, d.x, d.y, d.z, d.w};
#pragma unroll
                            for (int k = 16; k < 32; ++k)
                                if (k <= nh[u] && hit(g2[(k >> 1) - 8], k & 1)) tv[u] = 1;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        if (slotv[u] < 0) continue;
                        const int slot = slotv[u];
                        const int32_t l = (int32_t)cnts[slot];
                        int32_t t = tv[u];
                        if (nh[u] > 31) {
                            const int32_t j = jv[u];
                            const int32_t x0 = __ldg(&hoff[j]), x1 = __ldg(&hoff[j + 1]);
                            if (x1 - x0 <= bigk) {
                                // the partner's hubs against the row's bitmap, four at a time
                                for (int32_t y = x0; y < x1 && !t; y += 4) {
                                    int32_t hv[4];
#pragma unroll
                                    for (int v = 0; v < 4; ++v) hv[v] = y + v < x1 ? __ldg(&hlist[y + v]) : -1;
#pragma unroll
                                    for (int v = 0; v < 4; ++v)
                                        if (hv[v] >= 0 && ((hbits[hv[v] >> 5] >> (hv[v] & 31)) & 1u)) t = 1;
                                }
                            } else {
                                // the row's hubs against the partner's bitmap
                                const uint32_t* bb = bigbits + (int64_t)__ldg(&bigidx[j]) * HP_WORDS;
                                for (int32_t y = 0; y < ki && !t; y += 4) {
                                    uint32_t bw[4];
#pragma unroll
                                    for (int v = 0; v < 4; ++v)
                                        bw[v] = y + v < ki ? __ldg(&bb[hmine[y + v] >> 5]) : 0u;
#pragma unroll
                                    for (int v = 0; v < 4; ++v)
                                        if (y + v < ki && ((bw[v] >> (hmine[y + v] & 31)) & 1u)) t = 1;
                                }
                            }
                        }
                        const int32_t ov = l + t;
                        cnts[slot] = ov >= s ? (uint32_t)ov : 0u;
                    }
                }
                __syncthreads();
                int32_t mine = 0;
#pragma unroll
                for (int r = 0; r < HP_SLOTS_PER_THREAD; ++r) {
                    const int slot = r * NT + tid;
                    mine += cnts[slot] > 0u ? 1 : 0;
                    if (ENS4) {  // a survivor's count is its overlap (>= the first threshold)
                        const uint32_t ov = cnts[slot];
                        en0 += ov > 0u && ov >= es0 ? 1 : 0;
                        en1 += ov >= es1 ? 1 : 0;
                        en2 += ov >= es2 ? 1 : 0;
                        en3 += ov >= es3 ? 1 : 0;
                    }
                    if (!FILL && keys[slot] != HP_EMPTY) {  // the counting pass clears as it reads
                        keys[slot] = HP_EMPTY;
                        cnts[slot] = 0u;
                    }
                }
                int32_t c;
                const int32_t ex = block_excl_scan<NT>(mine, &c, tmp);
                if (!FILL) {
                    clean = true;
                } else if (c > 0) {
                    // survivors to the CTA's scratch list, then back into the table's
                    // memory in order of j: counted into HP_BUCKETS buckets by j,
                    // placed, and each thread sorts its buckets by insertion (a
                    // crowded bucket sends the whole list to a bitonic sort)
                    int32_t p = ex;
#pragma unroll
                    for (int r = 0; r < HP_SLOTS_PER_THREAD; ++r) {
                        const int slot = r * NT + tid;
                        const uint32_t ov = cnts[slot];
                        if (ov > 0u)
                            surv[p++] = ((unsigned long long)(uint32_t)keys[slot] << 32) | ov;
                    }
                    int32_t* hist = reinterpret_cast<int32_t*>(chk);  // HP_BUCKETS + 1
                    const int64_t a = sh_a, span = (int64_t)b - a;
                    for (int32_t t = tid; t <= HP_BUCKETS; t += NT) hist[t] = 0;
                    __syncthreads();
                    constexpr int SPT = HP_CAP / NT;  // survivors per thread, at most
                    int32_t bp[SPT];
#pragma unroll
                    for (int u = 0; u < SPT; ++u) {
                        const int32_t t = u * NT + tid;
                        if (t < c) {
                            const int32_t j = (int32_t)(surv[t] >> 32);
                            bp[u] = atomicAdd(&hist[(int32_t)(((int64_t)j - a) * HP_BUCKETS / span)], 1);
                        }
                    }
                    __syncthreads();
                    constexpr int BPT = HP_BUCKETS / NT;  // buckets per thread
                    int32_t hs[BPT], tot = 0;
#pragma unroll
                    for (int u = 0; u < BPT; ++u) {
                        hs[u] = hist[tid * BPT + u];
                        tot += hs[u];
                    }
                    int32_t all;
                    int32_t run = block_excl_scan<NT>(tot, &all, tmp);
                    const int32_t my0 = run;
#pragma unroll
                    for (int u = 0; u < BPT; ++u) {
                        hist[tid * BPT + u] = run;
                        run += hs[u];
                    }
                    __syncthreads();
#pragma unroll
                    for (int u = 0; u < SPT; ++u) {
                        const int32_t t = u * NT + tid;
                        if (t < c) {
                            const unsigned long long v = surv[t];
                            const int32_t j = (int32_t)(v >> 32);
                            sortbuf[hist[(int32_t)(((int64_t)j - a) * HP_BUCKETS / span)] + bp[u]] = v;
                        }
                    }
                    __syncthreads();
                    bool crowded = false;
                    {
                        int32_t st = my0;
                        for (int u = 0; u < BPT; ++u) {
                            const int32_t n = hs[u];
                            if (n > 32) {
                                crowded = true;
                            } else {
                                for (int32_t x = st + 1; x < st + n; ++x) {
                                    const unsigned long long v = sortbuf[x];
                                    int32_t y = x - 1;
                                    while (y >= st && sortbuf[y] > v) {
                                        sortbuf[y + 1] = sortbuf[y];
                                        --y;
                                    }
                                    sortbuf[y + 1] = v;
                                }
                            }
                            st += n;
                        }
                    }
                    if (__syncthreads_or(crowded)) {
                        int32_t P = 1;
                        while (P < c) P <<= 1;
                        for (int32_t t = c + tid; t < P; t += NT) sortbuf[t] = ~0ull;
                        __syncthreads();
                        for (int32_t k = 2; k <= P; k <<= 1) {
                            for (int32_t jj = k >> 1; jj > 0; jj >>= 1) {
                                for (int32_t t = tid; t < P; t += NT) {
                                    const int32_t u = t ^ jj;
                                    if (u > t) {
                                        const unsigned long long x = sortbuf[t], y = sortbuf[u];
                                        if ((x > y) == ((t & k) == 0)) {
                                            sortbuf[t] = y;
                                            sortbuf[u] = x;
                                        }
                                    }
                                }
                                __syncthreads();
                            }
                        }
                    }
                    for (int32_t t = tid; t < c; t += NT) {
                        const unsigned long long v = sortbuf[t];
                        const int64_t p2 = obase + out_pos + t;
                        if (p2 < olimit) {
                            if (stg) {
                                sa.J[p2] = (int32_t)(v >> 32) - ib;
                                sa.O[p2] = (uint8_t)(v & 0xffu);
                            } else {
                                I[p2] = i - ib;
                                J[p2] = (int32_t)(v >> 32) - ib;
                                O[p2] = (int32_t)(v & 0xffffffffu);
                            }
                        } else if (stg) {
                            sh_sovf = 1;  // the item is filled again later
                        } else {
                            atomicOr(err, ERR_BOUNDS);
                        }
                    }
                    clean = false;
                }
                out_pos += c;
            }
            if (ENS4) {
                int32_t t0c = 0, t1c = 0, t2c = 0, t3c = 0;
                block_excl_scan<NT>(en0, &t0c, tmp);
                block_excl_scan<NT>(en1, &t1c, tmp);
                block_excl_scan<NT>(en2, &t2c, tmp);
                block_excl_scan<NT>(en3, &t3c, tmp);
                if (tid == 0) {
                    const int32_t tc[4] = {t0c, t1c, t2c, t3c};
                    for (int32_t t = 0; t < eap->k; ++t) eap->icnt[t * eap->stride + qq] = tc[t];
                }
            } else if (!FILL && tid == 0) {
                icnt[qq] = (int32_t)out_pos;
            }
            if (stg && tid == 0) {
                icnt[qq] = (int32_t)out_pos;
                if (!sh_sovf) {
                    sa.at[qq] = obase;
                    sh_cpos = obase + out_pos;
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace

void hubpair_setup(int sms, int ctas[2]) {
    SLG_CUDA_TRY(cudaFuncSetAttribute(k_hubpair_items<false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HP_SMEM));
    for (int f = 0; f < 2; ++f) {
        auto kern = f ? k_hubpair_items<true> : k_hubpair_items<false>;
        SLG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)HP_SMEM));
        int d = 0;
        SLG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, kern, HP_THREADS, HP_SMEM));
        ctas[f] = sms * (d > 0 ? d : 1);
    }
}

void launch_hubpair(bool fill, int ctas, const GraphDev& g, const Plan& p, RowS rs,
                    int32_t item_lo, int32_t item_hi, int32_t* icnt, const int64_t* ioff,
                    int32_t* I, int32_t* J, int32_t* O, int32_t* queue, int64_t limit,
                    int32_t* err, cudaStream_t st, const StageArgs& sa, const EnsArgs* ens4) {
    const HubPairs& hp = *p.hp;
    int32_t* scratch = dalloc<int32_t>((size_t)ctas * HP_SCRATCH_WORDS, st);
    if (fill)
        k_hubpair_items<true><<<ctas, HP_THREADS, HP_SMEM, st>>>(
            p.items, p.mode_list[MODE_HUBPAIR], p.mode_rank[MODE_HUBPAIR], item_lo, item_hi,
            g.off, g.idx, p.wbeg, p.wend, p.idxTs, hp.hp_id, hp.hoff, hp.hlist, hp.bigidx,
            hp.bigbits, hp.hrec, hp.bigk, hp.off2, p.wbeg2, p.wend2, p.idxT2s, rs, icnt, ioff, I, J, O, queue,
            limit, err, scratch, sa, nullptr);
    else if (ens4)
        k_hubpair_items<false, true><<<ctas, HP_THREADS, HP_SMEM, st>>>(
            p.items, p.mode_list[MODE_HUBPAIR], p.mode_rank[MODE_HUBPAIR], item_lo, item_hi,
            g.off, g.idx, p.wbeg, p.wend, p.idxTs, hp.hp_id, hp.hoff, hp.hlist, hp.bigidx,
            hp.bigbits, hp.hrec, hp.bigk, hp.off2, p.wbeg2, p.wend2, p.idxT2s, rs, icnt, ioff, I, J, O, queue,
            limit, err, scratch, StageArgs{}, ens4);
    else
        k_hubpair_items<false><<<ctas, HP_THREADS, HP_SMEM, st>>>(
            p.items, p.mode_list[MODE_HUBPAIR], p.mode_rank[MODE_HUBPAIR], item_lo, item_hi,
            g.off, g.idx, p.wbeg, p.wend, p.idxTs, hp.hp_id, hp.hoff, hp.hlist, hp.bigidx,
            hp.bigbits, hp.hrec, hp.bigk, hp.off2, p.wbeg2, p.wend2, p.idxT2s, rs, icnt, ioff, I, J, O, queue,
            limit, err, scratch, StageArgs{}, nullptr);
    SLG_LAUNCH_CHECK();
    dfree(scratch, st);
}

}  // namespace slg
