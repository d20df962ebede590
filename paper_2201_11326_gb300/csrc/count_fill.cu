// Counting and filling: the inner loop of Algorithm 2 (Section III-C).
//
// For a row e_i and each of its vertices v_k, every later hyperedge e_j of
// adj(v_k) gets overlap_count[e_j] += 1; afterwards every e_j with count >= s
// is an s-incident partner. That is the "ikj" axpy order of Section III-B
// (for k in H^T.Adj[i], for j in H.Adj[k]: L[i,j] += 1) with the Boolean
// filter applied per row. The paper keeps the counts in a per-thread
// std::unordered_map; here a work item (row i, partners j in [jlo, jhi))
// keeps them on chip in one of these forms (the sparse accumulators, for rows
// spread thinly over a wide id range, are in sparse.cu):
//
//   MODE_WARP   one warp, a 256-slot open-addressing table in shared memory
//               (rows with at most 128 wedges, so the table never fills);
//   MODE_BLOCK  one CTA, a 4096-slot open-addressing table in shared memory
//               with atomicAdd counts; a slice with more than 2048 distinct
//               partners is split in two j halves and redone, so no table
//               overflows and nothing spills off chip;
//   MODE_DENSE  one CTA per slice walking 32768-wide j tiles in order: the
//               hub part of each overlap is a popcount of two 32-bit hub
//               masks, the rest direct-addressed 16-bit counters (see below);
//   MODE_WDENSE the same at warp granularity with 8-bit counters, for dense
//               rows with at most 32 non-hub wedge ranges.
//
// Both passes run the same code: the counting pass stores the number of
// partners per item, a scan turns those into output offsets, and the fill
// pass writes (i, j, overlap) in ascending j with warp-ballot compaction (the
// per-thread output lists of Algorithm 2 are not needed).
#include <cstdio>
#include <mutex>

#include "kernel_util.cuh"
#include "plan.cuh"

namespace slg {
namespace {

constexpr int32_t EMPTY = -1;
// Fibonacci hashing of a hyperedge id into a table of 2^(32-shift) slots.
__device__ __forceinline__ uint32_t slot_of(int32_t j, int shift) {
    return ((uint32_t)j * 2654435761u) >> shift;
}

// Insert-or-increment with linear probing. Keys go EMPTY -> j once and never
// change again, so a plain read that sees a key is final; a read that sees
// EMPTY is settled by the CAS. Returns 1 when this call created the key, 0
// when it existed, -1 when every slot was probed without finding room (the
// callers size their tables so that this cannot happen; the bound only
// guarantees that the loop ends).
__device__ __forceinline__ int table_add(int32_t* keys, int32_t* cnts, uint32_t mask, int shift,
                                         int32_t j) {
    uint32_t h = slot_of(j, shift);
    volatile int32_t* vk = keys;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const int32_t k = vk[h];
        if (k == j) {
            atomicAdd(&cnts[h], 1);
            return 0;
        }
        if (k == EMPTY) {
            const int32_t old = atomicCAS(&keys[h], EMPTY, j);
            if (old == EMPTY) {
                atomicAdd(&cnts[h], 1);
                return 1;
            }
            if (old == j) {
                atomicAdd(&cnts[h], 1);
                return 0;
            }
        }
        h = (h + 1) & mask;
    }
    return -1;
}

// Several thresholds in one counting launch (an ensemble, Algorithm 3): the
// counting pass counts every list's partners. (Each list is then filled by
// the single-threshold kernels.)

// ============================================================ MODE_WARP

template <bool FILL>
__global__ void __launch_bounds__(WARP_CTA_WARPS * 32)
k_warp_items(const Item* __restrict__ items, const int32_t* __restrict__ list,
             const int32_t* __restrict__ rank, int32_t item_lo, int32_t item_hi,
             const int32_t* __restrict__ off, const int32_t* __restrict__ wbeg,
             const int32_t* __restrict__ wend, const int32_t* __restrict__ idxTs, RowS rs,
             int32_t* __restrict__ icnt, const int64_t* __restrict__ ioff, int32_t* __restrict__ I,
             int32_t* __restrict__ J, int32_t* __restrict__ O, int64_t limit,
             int32_t* __restrict__ err) {
    constexpr int SHIFT = 32 - 8;  // 256 slots
    static_assert(WARP_TABLE == 256, "slot hash assumes 256 slots");
    __shared__ int32_t keys[WARP_CTA_WARPS][WARP_TABLE];
    __shared__ int32_t cnts[WARP_CTA_WARPS][WARP_TABLE];
    __shared__ int32_t pre[WARP_CTA_WARPS][33];
    __shared__ int32_t beg[WARP_CTA_WARPS][32];
    __shared__ int32_t sj[WARP_CTA_WARPS][WARP_TABLE / 2];
    __shared__ int32_t so[WARP_CTA_WARPS][WARP_TABLE / 2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int32_t lo = rank[item_lo], hi = rank[item_hi];
    for (int t = lane; t < WARP_TABLE; t += 32) {
        keys[w][t] = EMPTY;
        cnts[w][t] = 0;
    }
    __syncwarp();
    const int64_t nw = (int64_t)gridDim.x * WARP_CTA_WARPS;
    for (int64_t pos = lo + (int64_t)blockIdx.x * WARP_CTA_WARPS + w; pos < hi; pos += nw) {
        const int32_t q = list[pos];
        if (FILL && ioff[q + 1] == ioff[q]) continue;  // nothing to write
        const Item it = items[q];
        const int32_t i = it.row;
        const int32_t s = rs.s_of(i);
        const int32_t ib = rs.base_of(i);
        const int32_t e1 = off[i + 1];
        for (int32_t eb = off[i]; eb < e1; eb += 32) {
            const int32_t e = eb + lane;
            int32_t b = 0, len = 0;
            if (e < e1) {
                b = wbeg[e];
                len = wend[e] - b;
            }
            int32_t inc = len;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane >= d) inc += y;
            }
            pre[w][lane + 1] = inc;
            if (lane == 0) pre[w][0] = 0;
            beg[w][lane] = b;
            __syncwarp();
            const int32_t tot = pre[w][32];
            for (int32_t t = lane; t < tot; t += 32) {
                int32_t a = 0, z = 31;  // largest a with pre[a] <= t
                while (a < z) {
                    const int32_t mid = (a + z + 1) >> 1;
                    if (pre[w][mid] <= t)
                        a = mid;
                    else
                        z = mid - 1;
                }
                if (table_add(keys[w], cnts[w], WARP_TABLE - 1, SHIFT,
                              idxTs[beg[w][a] + t - pre[w][a]]) < 0)
                    atomicOr(err, ERR_TABLE);
            }
            __syncwarp();
        }
        // survivors, in slot order
        int32_t count = 0;
        for (int r = 0; r < WARP_TABLE / 32; ++r) {
            const int slot = r * 32 + lane;
            const int32_t k = keys[w][slot];
            const int32_t c = cnts[w][slot];
            const bool f = (k != EMPTY) && (c >= s);
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (FILL && f) {
                sj[w][count + __popc(bal & lt)] = k;
                so[w][count + __popc(bal & lt)] = c;
            }
            count += __popc(bal);
        }
        if (!FILL) {
            if (lane == 0) icnt[q] = count;
        } else {
            __syncwarp();
            const int64_t obase = ioff[q] - ioff[item_lo];
            for (int32_t t = lane; t < count; t += 32) {
                const int32_t jj = sj[w][t];
                int32_t r = 0;
                for (int32_t u = 0; u < count; ++u) r += (sj[w][u] < jj) ? 1 : 0;
                if (obase + r < limit) {
                    I[obase + r] = i - ib;
                    J[obase + r] = jj - ib;
                    O[obase + r] = so[w][t];
                } else {
                    atomicOr(err, ERR_BOUNDS);
                }
            }
        }
        __syncwarp();
        for (int t = lane; t < WARP_TABLE; t += 32) {
            keys[w][t] = EMPTY;
            cnts[w][t] = 0;
        }
        __syncwarp();
    }
}

// =========================================================== MODE_BLOCK

template <bool FILL>
__global__ void __launch_bounds__(BLOCK_THREADS)
k_block_items(const Item* __restrict__ items, const int32_t* __restrict__ list,
              const int32_t* __restrict__ rank, int32_t item_lo, int32_t item_hi,
              const int32_t* __restrict__ off, const int32_t* __restrict__ wbeg,
              const int32_t* __restrict__ wend, const int32_t* __restrict__ idxTs, RowS rs,
              int32_t* __restrict__ icnt, const int64_t* __restrict__ ioff,
              int32_t* __restrict__ I, int32_t* __restrict__ J, int32_t* __restrict__ O,
              int32_t* __restrict__ queue, int64_t limit, int32_t* __restrict__ err) {
    constexpr int NT = BLOCK_THREADS;
    constexpr int SHIFT = 32 - 12;  // 4096 slots
    static_assert(BLOCK_TABLE == 4096, "slot hash assumes 4096 slots");
    constexpr int SLOTS_PER_THREAD = BLOCK_TABLE / NT;
    __shared__ unsigned long long tab[BLOCK_TABLE];  // keys | counts, then the sort buffer
    __shared__ int32_t pre[NT + 1];
    __shared__ int32_t sub[NT];
    __shared__ int32_t stk_a[64], stk_b[64];
    __shared__ int32_t tmp[NT / 32 + 1];
    __shared__ int32_t sh_pos, sh_n, sh_a, sh_b;
    __shared__ volatile int32_t nkeys, ovf;
    int32_t* keys = reinterpret_cast<int32_t*>(tab);
    int32_t* cnts = keys + BLOCK_TABLE;
    const int tid = threadIdx.x;
    const int32_t lo = rank[item_lo], hi = rank[item_hi];

    for (;;) {
        if (tid == 0) sh_pos = lo + atomicAdd(queue, 1);
        __syncthreads();
        const int32_t pos = sh_pos;
        if (pos >= hi) break;
        const int32_t q = list[pos];
        if (FILL && ioff[q + 1] == ioff[q]) {  // nothing to write (same in every thread)
            __syncthreads();  // everyone has read sh_pos before thread 0 rewrites it
            continue;
        }
        const Item it = items[q];
        const int32_t i = it.row;
        const int32_t s = rs.s_of(i);
        const int32_t ib = rs.base_of(i);
        const int32_t e0 = off[i], e1 = off[i + 1];
        const int64_t obase = FILL ? ioff[q] - ioff[item_lo] : 0;
        int64_t out_pos = 0;  // same value in every thread
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
            for (int t = tid; t < BLOCK_TABLE; t += NT) {
                keys[t] = EMPTY;
                cnts[t] = 0;
            }
            __syncthreads();
            const int32_t a = sh_a, b = sh_b;
            for (int32_t eb = e0; eb < e1; eb += NT) {
                const int32_t e = eb + tid;
                int32_t lo_e = 0, len = 0;
                if (e < e1) {
                    const int32_t b0 = wbeg[e], t0 = wend[e];
                    if (t0 > b0) {
                        lo_e = lower_bound_dev(idxTs, b0, t0, a);
                        len = lower_bound_dev(idxTs, lo_e, t0, b) - lo_e;
                    }
                }
                int32_t total;
                const int32_t ex = block_excl_scan<NT>(len, &total, tmp);
                pre[tid] = ex;
                sub[tid] = lo_e;
                if (tid == 0) pre[NT] = total;
                __syncthreads();
                for (int32_t t = tid; t < total; t += NT) {
                    if (ovf) break;
                    int32_t x = 0, z = NT - 1;  // largest x with pre[x] <= t
                    while (x < z) {
                        const int32_t mid = (x + z + 1) >> 1;
                        if (pre[mid] <= t)
                            x = mid;
                        else
                            z = mid - 1;
                    }
                    const int32_t j = idxTs[sub[x] + t - pre[x]];
                    const int r = table_add(keys, cnts, BLOCK_TABLE - 1, SHIFT, j);
                    if (r > 0) {
                        if (atomicAdd((int32_t*)&nkeys, 1) >= BLOCK_CAP) ovf = 1;
                    } else if (r < 0) {
                        ovf = 1;  // no room: split, as for too many distinct keys
                    }
                }
                __syncthreads();
                if (ovf) break;
            }
            if (ovf) {
                // more distinct partners than the table may hold: redo as two halves
                if (tid == 0) {
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
            int32_t kk[SLOTS_PER_THREAD], cc[SLOTS_PER_THREAD];
            int32_t mine = 0;
#pragma unroll
            for (int r = 0; r < SLOTS_PER_THREAD; ++r) {
                const int slot = r * NT + tid;
                kk[r] = keys[slot];
                cc[r] = cnts[slot];
                mine += (kk[r] != EMPTY && cc[r] >= s) ? 1 : 0;
            }
            int32_t c;
            const int32_t ex = block_excl_scan<NT>(mine, &c, tmp);
            if (FILL && c > 0) {
                // the table has been read into registers: reuse it as the sort buffer
                int32_t p = ex;
#pragma unroll
                for (int r = 0; r < SLOTS_PER_THREAD; ++r)
                    if (kk[r] != EMPTY && cc[r] >= s)
                        tab[p++] = ((unsigned long long)(uint32_t)kk[r] << 32) | (uint32_t)cc[r];
                int32_t P = 1;
                while (P < c) P <<= 1;
                for (int32_t t = c + tid; t < P; t += NT) tab[t] = ~0ull;
                __syncthreads();
                for (int32_t k = 2; k <= P; k <<= 1) {
                    for (int32_t jj = k >> 1; jj > 0; jj >>= 1) {
                        for (int32_t t = tid; t < P; t += NT) {
                            const int32_t u = t ^ jj;
                            if (u > t) {
                                const unsigned long long x = tab[t], y = tab[u];
                                const bool up = (t & k) == 0;
                                if ((x > y) == up) {
                                    tab[t] = y;
                                    tab[u] = x;
                                }
                            }
                        }
                        __syncthreads();
                    }
                }
                for (int32_t t = tid; t < c; t += NT) {
                    const unsigned long long v = tab[t];
                    const int64_t p2 = obase + out_pos + t;
                    if (p2 < limit) {
                        I[p2] = i - ib;
                        J[p2] = (int32_t)(v >> 32) - ib;
                        O[p2] = (int32_t)(v & 0xffffffffu);
                    } else {
                        atomicOr(err, ERR_BOUNDS);
                    }
                }
            }
            out_pos += c;
            __syncthreads();
        }
        if (!FILL && tid == 0) icnt[q] = (int32_t)out_pos;
        __syncthreads();
    }
}

// =========================================================== MODE_DENSE
//
// Overlap of row i with partner j, split by vertex class:
//   |e_i ∩ e_j| = popc(hubmask[i] & hubmask[j])            (hub vertices)
//               + #{non-hub v in e_i ∩ e_j, wedge (i,v,j)} (counted here)
// Hubs are the (at most 32) highest-degree vertices, fixed at load time;
// hubmask[r] has bit b set when hub b is in e_r. Pruning needs no mask
// change: a partner with |e_j| < s has overlap <= |e_j| < s whatever is
// added. Only non-hub wedges touch shared memory: 16-bit counters for one
// 32768-wide j tile, incremented by atomicAdd with lane-contiguous reads of
// adj_s (consecutive lanes -> consecutive partners -> distinct banks). Each
// non-hub wedge range keeps a cursor that advances tile by tile (the lists are
// ascending), so no per-tile search is needed.

constexpr int HALF = DENSE_TILE / 2;  // 16-bit counters, two per word
constexpr int LOG_HALF = 14;
static_assert((1 << LOG_HALF) == HALF, "tile must be 2^15");
constexpr int DENSE_WARPS = DENSE_THREADS / 32;
constexpr int DENSE_SEG = DENSE_TILE / DENSE_WARPS;  // partners per warp per tile
static_assert(DENSE_SEG == 2048, "extraction keeps 64 ballots per warp");
constexpr size_t DENSE_SMEM = sizeof(uint32_t) * HALF + sizeof(int32_t) * 2 * DENSE_MAXE;

__device__ __forceinline__ int32_t dense_count(uint32_t hmi, const uint32_t* __restrict__ hubmask,
                                               const uint32_t* ctr, int32_t t0, int32_t ci) {
    const uint32_t w = ctr[ci & (HALF - 1)];
    return __popc(hmi & __ldg(&hubmask[t0 + ci])) +
           (int32_t)((w >> ((ci >> LOG_HALF) << 4)) & 0xffffu);
}

template <bool FILL, bool ENS>
__global__ void __launch_bounds__(DENSE_THREADS)
k_dense_items(const Item* __restrict__ items, const int32_t* __restrict__ list,
              const int32_t* __restrict__ rank, int32_t item_lo, int32_t item_hi,
              const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
              const int32_t* __restrict__ hubidx, const uint32_t* __restrict__ hubmask,
              const int32_t* __restrict__ wbeg, const int32_t* __restrict__ wend,
              const int32_t* __restrict__ idxTs, RowS rs, int32_t* __restrict__ icnt,
              const int64_t* __restrict__ ioff, int32_t* __restrict__ I, int32_t* __restrict__ J,
              int32_t* __restrict__ O, int32_t* __restrict__ queue, int64_t limit,
              int32_t* __restrict__ err, const EnsArgs ea) {
    constexpr int NT = DENSE_THREADS;
    constexpr int NW = DENSE_WARPS;
    extern __shared__ __align__(16) uint32_t dyn[];
    uint32_t* ctr = dyn;                                    // HALF words
    int32_t* cur = reinterpret_cast<int32_t*>(dyn + HALF);  // non-hub cursors
    int32_t* endp = cur + DENSE_MAXE;
    __shared__ int32_t wtot[NW];
    // ensemble: survivors of lists 1.. per warp segment of the current tile
    __shared__ int32_t wtot_e[ENS ? NW : 1][ENS ? ENS_MAX : 1];
    __shared__ int32_t sh_pos, sh_nnh;
    static_assert(!(FILL && ENS), "ensemble lists are filled one at a time");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int32_t lo = rank[item_lo], hi = rank[item_hi];

    for (;;) {
        if (tid == 0) {
            sh_pos = lo + atomicAdd(queue, 1);
            sh_nnh = 0;
        }
        __syncthreads();
        const int32_t pos = sh_pos;
        if (pos >= hi) break;
        const int32_t q = list[pos];
        if (FILL && ioff[q + 1] == ioff[q]) {  // nothing to write (same in every thread)
            __syncthreads();  // everyone has read sh_pos before thread 0 rewrites it
            continue;
        }
        const Item it = items[q];
        const int32_t i = it.row;
        const int32_t s = rs.s_of(i);
        const int32_t ib = rs.base_of(i);
        const uint32_t hmi = hubmask[i];
        const int32_t e0 = off[i];
        const int32_t ne = off[i + 1] - e0;
        // non-hub wedge ranges of the row, cursors at the item's first partner
        for (int32_t k = tid; k < ne; k += NT) {
            const int32_t e = e0 + k;
            const int32_t b0 = wbeg[e], t0 = wend[e];
            if (t0 > b0 && hubidx[idx[e]] < 0) {
                const int32_t c = (__ldg(&idxTs[b0]) >= it.jlo)
                                      ? b0 : lower_bound_dev(idxTs, b0, t0, it.jlo);
                if (c < t0) {
                    const int32_t slot = atomicAdd(&sh_nnh, 1);
                    cur[slot] = c;
                    endp[slot] = t0;
                }
            }
        }
        const int64_t obase = FILL ? ioff[q] - ioff[item_lo] : 0;
        int64_t out_pos = 0;
        // ensemble count: lane t (t >= 1) of every warp keeps list t's
        // survivors of the item so far
        int64_t ens_pos = 0;
        __syncthreads();
        const int32_t nnh = sh_nnh;
        for (int32_t t0 = it.jlo; t0 < it.jhi; t0 += DENSE_TILE) {
            const int32_t span = min(DENSE_TILE, it.jhi - t0);
            const int32_t t1 = t0 + span;
            const int32_t nz = span > HALF ? HALF : ((span + 3) & ~3);
            for (int32_t w = 4 * tid; w < nz; w += 4 * NT)
                *reinterpret_cast<uint4*>(ctr + w) = make_uint4(0, 0, 0, 0);
            __syncthreads();
            // non-hub wedges of this tile: one warp per wedge range, 32
            // consecutive entries per step, until a partner reaches t1
            for (int32_t k = warp; k < nnh; k += NW) {
                int32_t c = cur[k];
                const int32_t e = endp[k];
                for (;;) {
                    const int32_t p = c + lane;
                    const int32_t j = p < e ? __ldg(&idxTs[p]) : INT32_MAX;
                    const bool valid = j < t1;
                    if (valid) {
                        const int32_t ci = j - t0;
                        atomicAdd(&ctr[ci & (HALF - 1)], 1u << ((ci >> LOG_HALF) << 4));
                    }
                    const int n = __popc(__ballot_sync(0xffffffffu, valid));
                    c += n;
                    if (n < 32) break;
                }
                if (lane == 0) cur[k] = c;
            }
            __syncthreads();
            // extraction, pass 1: survivors per 32 partners, in j order per warp segment
            const int32_t seg0 = warp * DENSE_SEG;
            uint32_t bs0 = 0, bs1 = 0;
            int32_t cnt = 0, ecnt = 0;
            for (int32_t r = 0; r < DENSE_SEG / 32; ++r) {
                const int32_t ci = seg0 + r * 32 + lane;
                int32_t o = 0;
                if (ci < span) o = dense_count(hmi, hubmask, ctr, t0, ci);
                const bool f = ci < span && o >= s;
                const unsigned bal = __ballot_sync(0xffffffffu, f);
                if (FILL && lane == (r & 31)) {
                    if (r < 32)
                        bs0 = bal;
                    else
                        bs1 = bal;
                }
                cnt += __popc(bal);
                if (ENS && bal) {
                    // nested lists: the first list with no survivor ends the scan
                    for (int t = 1; t < ea.k; ++t) {
                        const unsigned bt = __ballot_sync(0xffffffffu, f && o >= ea.s[t]);
                        if (bt == 0) break;
                        if (lane == t) ecnt += __popc(bt);
                    }
                }
            }
            if (lane == 0) wtot[warp] = cnt;
            if (ENS && lane > 0 && lane < ea.k) wtot_e[warp][lane] = ecnt;
            __syncthreads();
            int32_t before = 0, tile_total = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const int32_t v = wtot[w];
                before += (w < warp) ? v : 0;
                tile_total += v;
            }
            int32_t etotal = 0;  // lane t: list t
            if (ENS && lane > 0 && lane < ea.k) {
#pragma unroll
                for (int w = 0; w < NW; ++w) etotal += wtot_e[w][lane];
            }
            if (FILL) {
                // pass 2: write survivors at their ordered positions
                int64_t base = obase + out_pos + before;
                for (int32_t r = 0; r < DENSE_SEG / 32; ++r) {
                    const unsigned bal = __shfl_sync(0xffffffffu, r < 32 ? bs0 : bs1, r & 31);
                    if (bal == 0) continue;
                    const bool mine = (bal >> lane) & 1u;
                    const int32_t ci = seg0 + r * 32 + lane;
                    int32_t o = 0;
                    if (mine) {
                        o = dense_count(hmi, hubmask, ctr, t0, ci);
                        const int64_t p2 = base + __popc(bal & lt);
                        if (p2 < limit) {
                            I[p2] = i - ib;
                            J[p2] = t0 + ci - ib;
                            O[p2] = o;
                        } else {
                            atomicOr(err, ERR_BOUNDS);
                        }
                    }
                    base += __popc(bal);
                }
            }
            out_pos += tile_total;
            if (ENS) ens_pos += etotal;
            __syncthreads();
        }
        if (!FILL && ENS) {
            if (tid == 0) ea.icnt[q] = (int32_t)out_pos;
            if (warp == 0 && lane > 0 && lane < ea.k) ea.icnt[lane * ea.stride + q] = (int32_t)ens_pos;
        } else if (!FILL && tid == 0) {
            icnt[q] = (int32_t)out_pos;
        }
        __syncthreads();
    }
}

// ========================================================== MODE_WDENSE
//
// The dense handler at warp granularity, for rows with at most 32 non-hub
// wedge ranges (almost every dense row): one warp owns a slice, a j tile of
// 4096 8-bit counters (CTAs of 12 warps: four per SM when counting, three
// when filling, whose ring takes more shared memory; 12-warp CTAs measured
// 1.4% faster than 16-warp ones) and one non-hub cursor per lane, so no
// CTA barrier is ever needed. A non-hub count is at most 32 and a hub count at
// most 32, so every overlap fits a byte below 128. Counter of partner t0 + c:
// byte c % 4 of word c / 4, so a lane's four consecutive partners share one
// word. Tiles start at multiples of 32 ids. Per tile:
//   1. clear the counters;
//   2. add the non-hub wedges: ranges with a partner inside the tile take
//      part in rounds; a round loads the next 32 entries of up to four ranges
//      at once, then counts the ones below the tile end;
//   3. extraction, four consecutive partners per lane: hub masks by 16-byte
//      loads, overlaps summed and compared four at a time inside one 32-bit
//      word (each byte stays below 128, so no carry crosses bytes). The
//      counting pass adds up the survivors. The fill pass appends them in j
//      order to a per-warp ring in shared memory and stores them in chunks of
//      32 that start on 128-byte boundaries of I (only the first chunk of a
//      slice is shorter), so every store is a full, aligned line.

constexpr int WD_TILE_FILL = 4096;
constexpr int WD_SLOTS = WD_MAXR / 32;  // non-hub cursors per lane
constexpr int WD_RING = 256;  // fill: survivors waiting for an aligned store
constexpr int WD_CBLK = 4;    // 128-partner blocks whose loads are issued together
constexpr int WD_GROUP = 4;   // non-hub ranges loaded together per round
constexpr size_t WD_STAGE_WORDS = 2 * WD_MAXR;  // cursor and end of each range
constexpr size_t wd_warp_words(bool fill) {
    return (fill ? WD_TILE_FILL / 4 + 2 * WD_RING : WD_TILE / 4) + WD_STAGE_WORDS;
}
constexpr size_t WD_SMEM = sizeof(uint32_t) * wd_warp_words(false) * WD_WARPS;
constexpr size_t WD_SMEM_FILL = sizeof(uint32_t) * wd_warp_words(true) * WD_WARPS;
static_assert(WD_TILE % (128 * WD_CBLK) == 0 && WD_TILE_FILL % (128 * WD_CBLK) == 0, "tiles");
static_assert(MAX_HUBS + WD_MAXR < 128, "byte-wise overlap sums must stay below 128");
static_assert(WD_MAXR % 32 == 0 && WD_SLOTS >= 1 && WD_SLOTS <= 2, "cursors per lane");

template <bool FILL, bool ENS>
__global__ void __launch_bounds__(WD_WARPS * 32, (FILL || ENS) ? 3 : 4)
k_wdense_items(const Item* __restrict__ items, const int32_t* __restrict__ list,
               const int32_t* __restrict__ rank, int32_t item_lo, int32_t item_hi,
               const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
               const int32_t* __restrict__ hubidx, const uint32_t* __restrict__ hubmask,
               const int32_t* __restrict__ wbeg, const int32_t* __restrict__ wend,
               const int32_t* __restrict__ idxTs, RowS rs, int32_t* __restrict__ icnt,
               const int64_t* __restrict__ ioff, int32_t* __restrict__ I,
               int32_t* __restrict__ J, int32_t* __restrict__ O, int32_t* __restrict__ queue,
               int64_t limit, int32_t* __restrict__ err, const EnsArgs ea) {
    constexpr int TILE = FILL ? WD_TILE_FILL : WD_TILE;
    constexpr int WORDS = TILE / 4;
    extern __shared__ __align__(16) uint32_t dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* ctr = dyn + (size_t)warp * wd_warp_words(FILL);
    int32_t* stage = reinterpret_cast<int32_t*>(ctr + WORDS);  // [0..63] cursor, [64..127] end
    int2* ring = reinterpret_cast<int2*>(stage + WD_STAGE_WORDS);  // fill only
    static_assert(!(FILL && ENS), "ensemble lists are filled one at a time");
    const unsigned lt = (1u << lane) - 1u;
    const int32_t lo = rank[item_lo], hi = rank[item_hi];

    for (;;) {
        int32_t pos = 0;
        if (lane == 0) pos = lo + atomicAdd(queue, 1);
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (pos >= hi) break;
        const int32_t q = list[pos];
        if (FILL && ioff[q + 1] == ioff[q]) continue;  // nothing to write
        const Item it = items[q];
        const int32_t i = it.row;
        const int32_t ib = rs.base_of(i);
        // byte-wise threshold: x >= s  <=>  bit 7 of x + (128 - s), for x < 128
        const uint32_t bias4 = 0x01010101u * (uint32_t)(128 - min(rs.s_of(i), 128));
        const uint32_t hmi = hubmask[i];
        const int32_t e0 = off[i];
        const int32_t ne = off[i + 1] - e0;
        // gather the non-hub wedge ranges, cursor at the slice's first partner
        int32_t nr = 0;
        for (int32_t kb = 0; kb < ne; kb += 32) {
            const int32_t k = kb + lane;
            bool ok = false;
            int32_t c = 0, t = 0;
            if (k < ne) {
                const int32_t e = e0 + k;
                const int32_t b0 = wbeg[e];
                t = wend[e];
                if (t > b0 && hubidx[idx[e]] < 0) {
                    c = (__ldg(&idxTs[b0]) >= it.jlo) ? b0 : lower_bound_dev(idxTs, b0, t, it.jlo);
                    ok = c < t;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, ok);
            const int32_t slot = nr + __popc(bal & lt);
            if (ok) {
                if (slot < WD_MAXR) {
                    stage[slot] = c;
                    stage[WD_MAXR + slot] = t;
                } else {
                    atomicOr(err, ERR_TABLE);  // binning guarantees <= 64 ranges
                }
            }
            nr += __popc(bal);
        }
        nr = min(nr, WD_MAXR);
        __syncwarp();
        // ranges lane, 32 + lane, ... (one per slot)
        int32_t cur[WD_SLOTS], end[WD_SLOTS], nxt[WD_SLOTS];
#pragma unroll
        for (int u = 0; u < WD_SLOTS; ++u) {
            const int32_t k = u * 32 + lane;
            cur[u] = k < nr ? stage[k] : 0;
            end[u] = k < nr ? stage[WD_MAXR + k] : 0;
            // partner at the cursor (INT32_MAX once the range is used up)
            nxt[u] = (k < nr && cur[u] < end[u]) ? __ldg(&idxTs[cur[u]]) : INT32_MAX;
        }
        __syncwarp();

        // ensemble count: lane t keeps list t's count
        int64_t ens_pos = 0;
        // fill: survivors collect in the ring and leave it in chunks that end
        // on 128-byte boundaries of I (the first chunk is shorter)
        int64_t wpos = FILL ? ioff[q] - ioff[item_lo] : 0;  // next output position
        int32_t rhead = 0, rcount = 0;
        int32_t need = FILL ? 32 - (int32_t)((reinterpret_cast<uintptr_t>(I + wpos) >> 2) & 31) : 32;
        int32_t my_count = 0;
        for (int32_t t0 = it.jlo & ~31; t0 < it.jhi; t0 += TILE) {
            const int32_t t1 = min(t0 + TILE, it.jhi);  // partners j in [max(t0, jlo), t1)
            const int32_t jfirst = max(t0, it.jlo);
            const int32_t span = t1 - t0;
            // 1. clear (only the words this tile uses)
            const int32_t nzw = (((span + 3) >> 2) + 3) & ~3;  // words, whole uint4s
            for (int32_t w = 4 * lane; w < nzw; w += 128)
                *reinterpret_cast<uint4*>(ctr + w) = make_uint4(0, 0, 0, 0);
            __syncwarp();
            // 2. non-hub wedges
            unsigned act[WD_SLOTS];
#pragma unroll
            for (int u = 0; u < WD_SLOTS; ++u) act[u] = __ballot_sync(0xffffffffu, nxt[u] < t1);
            auto any_active = [&]() {
                unsigned x = 0;
#pragma unroll
                for (int u = 0; u < WD_SLOTS; ++u) x |= act[u];
                return x != 0;
            };
            while (any_active()) {
                int32_t kk[WD_GROUP], vv[WD_GROUP];
                unsigned aa[WD_SLOTS];
#pragma unroll
                for (int u = 0; u < WD_SLOTS; ++u) aa[u] = act[u];
#pragma unroll
                for (int g = 0; g < WD_GROUP; ++g) {
                    int32_t k = -1;
#pragma unroll
                    for (int u = 0; u < WD_SLOTS; ++u) {
                        if (k < 0 && aa[u]) {
                            k = 32 * u + __ffs(aa[u]) - 1;
                            aa[u] &= aa[u] - 1u;
                        }
                    }
                    kk[g] = k;
                    int32_t cs = cur[0], es = end[0];
#pragma unroll
                    for (int u = 1; u < WD_SLOTS; ++u)
                        if ((k >> 5) == u) {
                            cs = cur[u];
                            es = end[u];
                        }
                    const int32_t c = __shfl_sync(0xffffffffu, cs, k & 31);
                    const int32_t e = __shfl_sync(0xffffffffu, es, k & 31);
                    const int32_t p = c + lane;
                    vv[g] = (k >= 0 && p < e) ? __ldg(&idxTs[p]) : INT32_MAX;
                }
#pragma unroll
                for (int g = 0; g < WD_GROUP; ++g) {
                    const int32_t k = kk[g];
                    if (k < 0) break;
                    const bool valid = vv[g] < t1;
                    if (valid) {
                        const int32_t ci = vv[g] - t0;
                        atomicAdd(&ctr[ci >> 2], 1u << ((ci & 3) << 3));
                    }
                    const int n = __popc(__ballot_sync(0xffffffffu, valid));
                    // the first entry not taken is the range's next partner
                    const int32_t nx = __shfl_sync(0xffffffffu, vv[g], n & 31);
                    const int uk = k >> 5;
#pragma unroll
                    for (int u = 0; u < WD_SLOTS; ++u) {
                        if (u != uk) continue;
                        if (lane == (k & 31)) {
                            cur[u] += n;
                            if (n < 32) nxt[u] = nx;
                        }
                        if (n < 32) act[u] &= ~(1u << (k & 31));
                    }
                }
            }
            __syncwarp();
            // 3. extraction: four consecutive partners per lane
            // (ensemble count: at most 128 partners per lane and tile, so a
            // byte holds each list's count until the tile ends)
            uint32_t ecnt[ENS ? ENS_MAX / 4 : 1];
#pragma unroll
            for (int u = 0; u < (ENS ? ENS_MAX / 4 : 1); ++u) ecnt[u] = 0;
            for (int32_t g = 0; g < span; g += 128 * WD_CBLK) {
                uint4 hv[WD_CBLK];
                uint32_t cw[WD_CBLK];
#pragma unroll
                for (int b = 0; b < WD_CBLK; ++b) {
                    const int32_t ci = g + b * 128 + 4 * lane;
                    if (ci < span) {
                        hv[b] = __ldg(reinterpret_cast<const uint4*>(hubmask + t0 + ci));
                        cw[b] = ctr[ci >> 2];
                    } else {
                        hv[b] = make_uint4(0, 0, 0, 0);
                        cw[b] = 0;
                    }
                }
#pragma unroll
                for (int b = 0; b < WD_CBLK; ++b) {
                    const int32_t ci = g + b * 128 + 4 * lane;
                    const uint32_t p4 = (uint32_t)__popc(hmi & hv[b].x) |
                                        ((uint32_t)__popc(hmi & hv[b].y) << 8) |
                                        ((uint32_t)__popc(hmi & hv[b].z) << 16) |
                                        ((uint32_t)__popc(hmi & hv[b].w) << 24);
                    const uint32_t c4 = p4 + cw[b];  // four overlaps, one per byte
                    uint32_t f4 = (c4 + bias4) & 0x80808080u;
                    uint32_t vmask = 0x80808080u;  // ensemble: the partners of this slice
                    const int32_t j0 = t0 + ci;
                    if (j0 < jfirst || j0 + 4 > t1) {  // partial block at a tile edge
#pragma unroll
                        for (int r = 0; r < 4; ++r)
                            if (j0 + r < jfirst || j0 + r >= t1) {
                                f4 &= ~(0x80u << (8 * r));
                                vmask &= ~(0x80u << (8 * r));
                            }
                    }
                    if (!FILL && ENS) {
                        // byte t % 4 of ecnt[t / 4]: list t's survivors of this tile
#pragma unroll
                        for (int t = 0; t < ENS_MAX; ++t)
                            if (t < ea.k)
                                ecnt[t >> 2] += (uint32_t)__popc((c4 + ea.bias[t]) & vmask)
                                                << (8 * (t & 3));
                        continue;
                    }
                    if (!FILL) {
                        my_count += __popc(f4);
                        continue;
                    }
                    const int32_t mine = __popc(f4);
                    int32_t inc = mine;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const int32_t y = __shfl_up_sync(0xffffffffu, inc, d);
                        if (lane >= d) inc += y;
                    }
                    const int32_t tot = __shfl_sync(0xffffffffu, inc, 31);
                    if (tot == 0) continue;
                    int32_t slot = rhead + rcount + inc - mine;
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        if ((f4 >> (8 * r + 7)) & 1u) {
                            ring[slot & (WD_RING - 1)] =
                                make_int2(j0 + r, (int32_t)((c4 >> (8 * r)) & 0xffu));
                            ++slot;
                        }
                    }
                    rcount += tot;
                    __syncwarp();
                    while (rcount >= need) {
                        if (lane < need) {
                            const int2 e = ring[(rhead + lane) & (WD_RING - 1)];
                            const int64_t p2 = wpos + lane;
                            if (p2 < limit) {
                                I[p2] = i - ib;
                                J[p2] = e.x - ib;
                                O[p2] = e.y;
                            } else {
                                atomicOr(err, ERR_BOUNDS);
                            }
                        }
                        rhead = (rhead + need) & (WD_RING - 1);
                        rcount -= need;
                        wpos += need;
                        need = 32;
                    }
                    __syncwarp();
                }
            }
            if (!FILL && ENS) {
#pragma unroll
                for (int t = 0; t < ENS_MAX; ++t) {
                    if (t >= ea.k) break;
                    const uint32_t tot =
                        __reduce_add_sync(0xffffffffu, (ecnt[t >> 2] >> (8 * (t & 3))) & 0xffu);
                    if (lane == t) ens_pos += tot;
                }
            }
            __syncwarp();
        }
        if (FILL && rcount > 0) {  // the slice's last, partial chunk
            if (lane < rcount) {
                const int2 e = ring[(rhead + lane) & (WD_RING - 1)];
                const int64_t p2 = wpos + lane;
                if (p2 < limit) {
                    I[p2] = i - ib;
                    J[p2] = e.x - ib;
                    O[p2] = e.y;
                } else {
                    atomicOr(err, ERR_BOUNDS);
                }
            }
            __syncwarp();
        }
        if (!FILL && ENS) {
            if (lane < ea.k) ea.icnt[lane * ea.stride + q] = (int32_t)ens_pos;
        } else if (!FILL) {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) my_count += __shfl_xor_sync(0xffffffffu, my_count, d);
            if (lane == 0) icnt[q] = my_count;
        }
    }
}

// =============================================================== digest

// Digest of a window: the pair at window position p belongs to the row whose
// output range holds base + p. For a single graph that row is I[p]; in a
// batch I holds graph-local ids, so the row is found by binary search over the
// window's row offsets, and the hash uses the local ids (so that each graph's
// digests equal those of the graph computed alone).
__global__ void k_digest(const int32_t* __restrict__ I, const int32_t* __restrict__ J,
                         const int32_t* __restrict__ O, int64_t P, int64_t base,
                         const int64_t* __restrict__ rowoff, int32_t r0, int32_t r1, RowS rs,
                         unsigned long long* __restrict__ total,
                         unsigned long long* __restrict__ rows, int32_t* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    unsigned long long acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < P; b += stride) {
        const int64_t p = b + threadIdx.x;
        bool ok = p < P;
        int32_t g = -1;  // global row
        unsigned long long h = 0;
        if (ok) {
            const int32_t li = I[p];
            if (rs.rbase) {
                int32_t a = r0, z = r1 - 1;  // last row with rowoff[row] <= base + p
                while (a < z) {
                    const int32_t mid = (a + z + 1) >> 1;
                    if (rowoff[mid] <= base + p)
                        a = mid;
                    else
                        z = mid - 1;
                }
                g = a;
                if (li != g - rs.rbase[g]) g = -2;
            } else {
                g = li;
            }
            if (g < r0 || g >= r1) {
                atomicOr(err, ERR_DIGEST);
                ok = false;
                g = -1;
            } else {
                h = pair_digest(li, base + p - rowoff[g], J[p], O[p]);
                acc += h;
            }
        }
        if (rows) {
            const unsigned peers = __match_any_sync(0xffffffffu, g);
            unsigned long long sum = 0;
            // sum of h over the peers, by shuffling each peer's value to the leader
            for (unsigned m2 = peers; m2; m2 &= m2 - 1) {
                const int src = __ffs(m2) - 1;
                sum += __shfl_sync(peers, h, src);
            }
            if (ok && lane == __ffs(peers) - 1) atomicAdd(&rows[g - r0], sum);
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if (lane == 0 && acc) atomicAdd(total, acc);
}

struct Occupancy {
    int sms = 0;
    int warp_ctas = 0, block_ctas = 0, dense_ctas = 0, sparse_ctas[2] = {}, wsparse_ctas[2] = {};
    int hubpair_ctas[2] = {};
    int wdense_ctas[2][2] = {};  // [fill][ensemble]
};

Occupancy g_occ;
std::once_flag g_occ_once;

template <bool FILL, bool ENS>
int wdense_setup(int sms) {
    const size_t smem = FILL ? WD_SMEM_FILL : WD_SMEM;
    SLG_CUDA_TRY(cudaFuncSetAttribute(k_wdense_items<FILL, ENS>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int d = 0;
    SLG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, k_wdense_items<FILL, ENS>,
                                                               WD_WARPS * 32, smem));
    return sms * (d > 0 ? d : 1);
}

void occupancy_init() {
    Occupancy& o = g_occ;
    int dev = 0;
    SLG_CUDA_TRY(cudaGetDevice(&dev));
    SLG_CUDA_TRY(cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev));
    SLG_CUDA_TRY(cudaFuncSetAttribute(k_dense_items<false, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)DENSE_SMEM));
    SLG_CUDA_TRY(cudaFuncSetAttribute(k_dense_items<true, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)DENSE_SMEM));
    SLG_CUDA_TRY(cudaFuncSetAttribute(k_dense_items<false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)DENSE_SMEM));
    sparse_setup(o.sms, o.sparse_ctas);
    wsparse_setup(o.sms, o.wsparse_ctas);
    hubpair_setup(o.sms, o.hubpair_ctas);
    o.wdense_ctas[0][0] = wdense_setup<false, false>(o.sms);
    o.wdense_ctas[1][0] = wdense_setup<true, false>(o.sms);
    o.wdense_ctas[0][1] = wdense_setup<false, true>(o.sms);
    int a = 0, b = 0, c = 0;
    SLG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_warp_items<true>,
                                                               WARP_CTA_WARPS * 32, 0));
    SLG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_block_items<true>,
                                                               BLOCK_THREADS, 0));
    SLG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_dense_items<true, false>,
                                                               DENSE_THREADS, DENSE_SMEM));
    o.warp_ctas = o.sms * (a > 0 ? a : 1);
    o.block_ctas = o.sms * (b > 0 ? b : 1);
    o.dense_ctas = o.sms * (c > 0 ? c : 1);
}

Occupancy& occupancy() {
    std::call_once(g_occ_once, occupancy_init);
    return g_occ;
}

constexpr unsigned ALL_MODES = (1u << NMODES) - 1u;
// ensemble counting launches: handlers with a fused form, and those run once
// per list
constexpr unsigned ENS_FUSED = (1u << MODE_DENSE) | (1u << MODE_WDENSE);
constexpr unsigned ENS_PER_LIST = ALL_MODES & ~ENS_FUSED;

// One launch per handler in `modes` that has items. queue: NMODES work-queue
// heads (zeroed, used once); err: the shared error flag. With `ea` (counting
// pass only), the dense handlers run their ensemble form (every list in one
// launch).
// Staged items of [item_lo, item_hi) into place, one warp per item: the item's
// staged pairs at[q] .. at[q] + n - 1 of the pool (n from the staged list's
// offsets st_ioff) go, in order, to ioff[q] - ioff[item_lo] onwards.
__global__ void k_place_staged(const Item* __restrict__ items, const int64_t* __restrict__ at,
                               const int64_t* __restrict__ st_ioff,
                               const int64_t* __restrict__ ioff, int32_t item_lo, int32_t item_hi,
                               const int32_t* __restrict__ sJ, const uint8_t* __restrict__ sO,
                               RowS rs, int32_t* __restrict__ I, int32_t* __restrict__ J,
                               int32_t* __restrict__ O, int64_t limit, int32_t* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t o0 = ioff[item_lo];
    for (int64_t q = item_lo + warp; q < item_hi; q += nwarps) {
        const int64_t a = at[q];
        if (a < 0) continue;
        const int64_t base = ioff[q] - o0, n = st_ioff[q + 1] - st_ioff[q];
        const int32_t i = items[q].row;
        const int32_t row = i - rs.base_of(i);
        int64_t w = base;  // next output position (same in every lane)
        for (int64_t k0 = 0; k0 < n; k0 += 32) {
            const int64_t k = k0 + lane;
            int32_t jv = 0, ov = 0;
            if (k < n) {
                jv = sJ[a + k];
                ov = (int32_t)sO[a + k];
            }
            const bool keep = k < n;
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int64_t p = w + __popc(bal & lt);
                if (p < limit) {
                    I[p] = row;
                    J[p] = jv;
                    O[p] = ov;
                } else {
                    atomicOr(err, ERR_BOUNDS);
                }
            }
            w += __popc(bal);
        }
        // the kept pairs are exactly the item's count in the list
        if (lane == 0 && w - base != ioff[q + 1] - ioff[q]) atomicOr(err, ERR_BOUNDS);
    }
}

// A list of an ensemble from the list before it: the lists are nested and in
// the same (i, j) order, so list t is list t-1's pairs with overlap >= s, in
// order. Blocks of FT_N = 4096 pairs: counted, scanned, then written.
constexpr int FT_THREADS = 256;
constexpr int FT_STEPS = 16;
constexpr int64_t FT_N = (int64_t)FT_THREADS * FT_STEPS;

__global__ void k_filter_count(const int32_t* __restrict__ O, int64_t n, int32_t s,
                               int32_t* __restrict__ counts) {
    __shared__ int32_t wsum[FT_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * FT_N;
    int32_t c = 0;
#pragma unroll
    for (int u = 0; u < FT_STEPS; ++u) {
        const int64_t x = base + u * FT_THREADS + tid;
        c += (x < n && O[x] >= s) ? 1 : 0;
    }
    c = (int32_t)__reduce_add_sync(0xffffffffu, (unsigned)c);
    if (lane == 0) wsum[warp] = c;
    __syncthreads();
    if (tid == 0) {
        int32_t t = 0;
        for (int w = 0; w < FT_THREADS / 32; ++w) t += wsum[w];
        counts[blockIdx.x] = t;
    }
}

__global__ void k_filter_write(const int32_t* __restrict__ I, const int32_t* __restrict__ J,
                               const int32_t* __restrict__ O, int64_t n, int32_t s,
                               const int64_t* __restrict__ boff, int32_t* __restrict__ I2,
                               int32_t* __restrict__ J2, int32_t* __restrict__ O2,
                               int64_t limit, int32_t* __restrict__ err) {
    constexpr int NW = FT_THREADS / 32;
    __shared__ int32_t at[FT_STEPS][NW];  // kept pairs before (step, warp), in pair order
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * FT_N;
    unsigned bal[FT_STEPS];
#pragma unroll
    for (int u = 0; u < FT_STEPS; ++u) {
        const int64_t x = base + u * FT_THREADS + tid;
        bal[u] = __ballot_sync(0xffffffffu, x < n && O[x] >= s);
        if (lane == 0) at[u][warp] = __popc(bal[u]);
    }
    __syncthreads();
    if (tid == 0) {  // pair order is step-major, then warp
        int32_t run = 0;
        for (int u = 0; u < FT_STEPS; ++u)
            for (int w = 0; w < NW; ++w) {
                const int32_t v = at[u][w];
                at[u][w] = run;
                run += v;
            }
    }
    __syncthreads();
    const int64_t o0 = boff[blockIdx.x];
#pragma unroll
    for (int u = 0; u < FT_STEPS; ++u) {
        if (!((bal[u] >> lane) & 1u)) continue;
        const int64_t x = base + u * FT_THREADS + tid;
        const int64_t p = o0 + at[u][warp] + __popc(bal[u] & lt);
        if (p < limit) {
            I2[p] = I[x];
            J2[p] = J[x];
            O2[p] = O[x];
        } else {
            atomicOr(err, ERR_BOUNDS);
        }
    }
}

template <bool FILL>
void launch_items(const GraphDev& g, const Plan& p, RowS rs, int32_t item_lo, int32_t item_hi,
                  int32_t* icnt, const int64_t* ioff, int32_t* I, int32_t* J, int32_t* O,
                  int64_t limit, int32_t* queue, int32_t* err, ModeTimer* mt, cudaStream_t st,
                  unsigned modes = ALL_MODES, const EnsArgs* ea = nullptr,
                  const StageArgs& sa = StageArgs{}, const EnsArgs* ens4 = nullptr) {
    Occupancy& oc = occupancy();
    const bool timed = mt && mt->on;
    const int pass = FILL && sa.J == nullptr ? 1 : 0;  // staging fills count as counting
    auto tick = [&](int mode, int edge) {
        if (timed) SLG_CUDA_TRY(cudaEventRecord(mt->ev[2 * mode + edge], st));
    };
    auto want = [&](int mode) { return ((modes >> mode) & 1u) && p.mode_count[mode] > 0; };
    bool ran[NMODES] = {};
    if (want(MODE_WARP)) {
        ran[MODE_WARP] = true;
        tick(MODE_WARP, 0);
        k_warp_items<FILL><<<oc.warp_ctas, WARP_CTA_WARPS * 32, 0, st>>>(
            p.items, p.mode_list[MODE_WARP], p.mode_rank[MODE_WARP], item_lo, item_hi, g.off,
            p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I, J, O, limit, err);
        SLG_LAUNCH_CHECK();
        tick(MODE_WARP, 1);
    }
    if (want(MODE_BLOCK)) {
        ran[MODE_BLOCK] = true;
        tick(MODE_BLOCK, 0);
        k_block_items<FILL><<<oc.block_ctas, BLOCK_THREADS, 0, st>>>(
            p.items, p.mode_list[MODE_BLOCK], p.mode_rank[MODE_BLOCK], item_lo, item_hi, g.off,
            p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I, J, O, queue + MODE_BLOCK, limit, err);
        SLG_LAUNCH_CHECK();
        tick(MODE_BLOCK, 1);
    }
    if (want(MODE_DENSE)) {
        ran[MODE_DENSE] = true;
        tick(MODE_DENSE, 0);
        if (ea) {
            if constexpr (!FILL)
                k_dense_items<false, true><<<oc.dense_ctas, DENSE_THREADS, DENSE_SMEM, st>>>(
                    p.items, p.mode_list[MODE_DENSE], p.mode_rank[MODE_DENSE], item_lo, item_hi,
                    g.off, g.idx, g.hubidx, g.hubmask, p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I,
                    J, O, queue + MODE_DENSE, limit, err, *ea);
        } else {
            k_dense_items<FILL, false><<<oc.dense_ctas, DENSE_THREADS, DENSE_SMEM, st>>>(
                p.items, p.mode_list[MODE_DENSE], p.mode_rank[MODE_DENSE], item_lo, item_hi,
                g.off, g.idx, g.hubidx, g.hubmask, p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I, J,
                O, queue + MODE_DENSE, limit, err, EnsArgs{});
        }
        SLG_LAUNCH_CHECK();
        tick(MODE_DENSE, 1);
    }
    if (want(MODE_WDENSE)) {
        ran[MODE_WDENSE] = true;
        tick(MODE_WDENSE, 0);
        const size_t smem = FILL ? WD_SMEM_FILL : WD_SMEM;
        if (ea) {
            if constexpr (!FILL)
                k_wdense_items<false, true><<<oc.wdense_ctas[0][1], WD_WARPS * 32, smem, st>>>(
                    p.items, p.mode_list[MODE_WDENSE], p.mode_rank[MODE_WDENSE], item_lo, item_hi,
                    g.off, g.idx, g.hubidx, g.hubmask, p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I,
                    J, O, queue + MODE_WDENSE, limit, err, *ea);
        } else {
            k_wdense_items<FILL, false><<<oc.wdense_ctas[FILL][0], WD_WARPS * 32, smem, st>>>(
                p.items, p.mode_list[MODE_WDENSE], p.mode_rank[MODE_WDENSE], item_lo, item_hi,
                g.off, g.idx, g.hubidx, g.hubmask, p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I, J,
                O, queue + MODE_WDENSE, limit, err, EnsArgs{});
        }
        SLG_LAUNCH_CHECK();
        tick(MODE_WDENSE, 1);
    }
    if (want(MODE_SPARSE)) {
        ran[MODE_SPARSE] = true;
        tick(MODE_SPARSE, 0);
        launch_sparse(FILL, oc.sparse_ctas[FILL], g, p, rs, item_lo, item_hi, icnt, ioff, I, J, O,
                      queue + MODE_SPARSE, limit, err, st, sa, ens4);
        tick(MODE_SPARSE, 1);
    }
    if (want(MODE_WSPARSE)) {
        ran[MODE_WSPARSE] = true;
        tick(MODE_WSPARSE, 0);
        launch_wsparse(FILL, oc.wsparse_ctas[FILL], g, p, rs, item_lo, item_hi, icnt, ioff, I, J,
                       O, queue + MODE_WSPARSE, limit, err, st);
        tick(MODE_WSPARSE, 1);
    }
    if (want(MODE_HUBPAIR) && p.hp) {
        ran[MODE_HUBPAIR] = true;
        tick(MODE_HUBPAIR, 0);
        launch_hubpair(FILL, oc.hubpair_ctas[FILL], g, p, rs, item_lo, item_hi, icnt, ioff, I, J,
                       O, queue + MODE_HUBPAIR, limit, err, st, sa, ens4);
        tick(MODE_HUBPAIR, 1);
    }
    if (timed) {
        for (int k = 0; k < NMODES; ++k) {
            if (!ran[k]) continue;
            float ms = 0;
            SLG_CUDA_TRY(cudaEventSynchronize(mt->ev[2 * k + 1]));
            SLG_CUDA_TRY(cudaEventElapsedTime(&ms, mt->ev[2 * k], mt->ev[2 * k + 1]));
            mt->ms[pass][k] += ms;
            mt->launches[pass][k] += 1;
        }
    }
}

// Device scratch: nq work-queue heads, then the error flag (all zero).
int32_t* new_scratch(cudaStream_t st, int nq = NMODES) {
    int32_t* s = nullptr;
    SLG_CUDA_TRY(cudaMallocAsync((void**)&s, sizeof(int32_t) * (nq + 1), st));
    SLG_CUDA_TRY(cudaMemsetAsync(s, 0, sizeof(int32_t) * (nq + 1), st));
    return s;
}

// Reads the error flag (synchronises) and frees the scratch.
void check_scratch(int32_t* s, cudaStream_t st, const char* what, int nq = NMODES) {
    int32_t e = 0;
    SLG_CUDA_TRY(cudaMemcpyAsync(&e, s + nq, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    SLG_CUDA_TRY(cudaFreeAsync(s, st));
    if (e) {
        char buf[128];
        snprintf(buf, sizeof(buf), "%s: device consistency check failed (flags %d)", what, e);
        throw Error{SLG_EINTERNAL, buf};
    }
}

EnsArgs ens_args(const Plan& p) {
    EnsArgs ea;
    ea.k = p.ens.k;
    for (int t = 0; t < ea.k; ++t) {
        ea.s[t] = p.ens.s[t];
        // byte-wise threshold: x >= s  <=>  bit 7 of x + (128 - s), for x < 128
        ea.bias[t] = 0x01010101u * (uint32_t)(128 - (p.ens.s[t] < 128 ? p.ens.s[t] : 128));
    }
    return ea;
}

}  // namespace

void run_count(const GraphDev& g, const Plan& p, RowS rs, int32_t* icnt, ModeTimer* mt,
               cudaStream_t st) {
    int32_t* sc = new_scratch(st);
    if (p.stage_at && p.stage_cap > 0) {
        // sparse-accumulator and hub-pair items: their fill kernels count and
        // stage while the pool lasts; the counting kernels below go on from
        // where each of their queues stopped
        SLG_CUDA_TRY(cudaMemsetAsync(p.stage_at, 0xff, sizeof(int64_t) * p.nitems, st));
        SLG_CUDA_TRY(cudaMemsetAsync(p.stage_cursor, 0, sizeof(unsigned long long), st));
        launch_items<true>(g, p, rs, 0, (int32_t)p.nitems, icnt, nullptr, nullptr, nullptr,
                           nullptr, 0, sc, sc + NMODES, mt, st,
                           (1u << MODE_SPARSE) | (1u << MODE_HUBPAIR), nullptr, p.stage_args());
    }
    launch_items<false>(g, p, rs, 0, (int32_t)p.nitems, icnt, nullptr, nullptr, nullptr, nullptr,
                        0, sc, sc + NMODES, mt, st);
    check_scratch(sc, st, "counting pass");
}

void run_count_modes(const GraphDev& g, const Plan& p, RowS rs, unsigned modes, int32_t* icnt,
                     ModeTimer* mt, cudaStream_t st) {
    int32_t* sc = new_scratch(st);
    launch_items<false>(g, p, rs, 0, (int32_t)p.nitems, icnt, nullptr, nullptr, nullptr, nullptr,
                        0, sc, sc + NMODES, mt, st, modes & ALL_MODES);
    check_scratch(sc, st, "counting pass");
}

void run_count_staged(const GraphDev& g, const Plan& p, RowS rs, int32_t item_lo, int32_t item_hi,
                      int32_t* icnt, ModeTimer* mt, cudaStream_t st) {
    if (item_hi <= item_lo) return;
    constexpr unsigned STAGED = (1u << MODE_SPARSE) | (1u << MODE_HUBPAIR);
    int32_t* sc = new_scratch(st);
    if (p.stage_at && p.stage_cap > 0) {
        SLG_CUDA_TRY(cudaMemsetAsync(p.stage_at + item_lo, 0xff,
                                     sizeof(int64_t) * (size_t)(item_hi - item_lo), st));
        SLG_CUDA_TRY(cudaMemsetAsync(p.stage_cursor, 0, sizeof(unsigned long long), st));
        launch_items<true>(g, p, rs, item_lo, item_hi, icnt, nullptr, nullptr, nullptr, nullptr, 0,
                           sc, sc + NMODES, mt, st, STAGED, nullptr, p.stage_args());
    }
    launch_items<false>(g, p, rs, item_lo, item_hi, icnt, nullptr, nullptr, nullptr, nullptr, 0,
                        sc, sc + NMODES, mt, st, STAGED);
    check_scratch(sc, st, "counting pass");
}

void run_fill(const GraphDev& g, const Plan& p, RowS rs, const int64_t* ioff, int32_t item_lo,
              int32_t item_hi, int32_t* I, int32_t* J, int32_t* O, int64_t limit, ModeTimer* mt,
              cudaStream_t st, StageUse su) {
    if (item_hi <= item_lo) return;
    int32_t* sc = new_scratch(st);
    StageArgs skip{};
    if (su.st_ioff && p.stage_at && p.stage_cap > 0) {
        // staged items are copied into place; the fill kernels skip them
        k_place_staged<<<152 * 16, 256, 0, st>>>(p.items, p.stage_at, su.st_ioff, ioff,
                                                 item_lo, item_hi, p.stage_J, p.stage_O, rs, I, J,
                                                 O, limit, sc + NMODES);
        SLG_LAUNCH_CHECK();
        skip.at = p.stage_at;
    }
    launch_items<true>(g, p, rs, item_lo, item_hi, nullptr, ioff, I, J, O, limit, sc, sc + NMODES,
                       mt, st, ALL_MODES, nullptr, skip);
    check_scratch(sc, st, "fill pass");
}

void run_filter(const int32_t* I, const int32_t* J, const int32_t* O, int64_t n, int32_t s,
                int32_t* I2, int32_t* J2, int32_t* O2, int64_t expect, cudaStream_t st) {
    if (n <= 0) {
        if (expect != 0) throw Error{SLG_EINTERNAL, "list filter: pairs expected from nothing"};
        return;
    }
    const int64_t nb = (n + FT_N - 1) / FT_N;
    int32_t* counts = dalloc<int32_t>((size_t)nb, st);
    int64_t* boff = dalloc<int64_t>((size_t)nb + 1, st);
    int32_t* sc = new_scratch(st);
    k_filter_count<<<(unsigned)nb, FT_THREADS, 0, st>>>(O, n, s, counts);
    SLG_LAUNCH_CHECK();
    scan_i32_to_i64(counts, boff, nb, st);
    k_filter_write<<<(unsigned)nb, FT_THREADS, 0, st>>>(I, J, O, n, s, boff, I2, J2, O2, expect,
                                                        sc + NMODES);
    SLG_LAUNCH_CHECK();
    int64_t got = 0;
    SLG_CUDA_TRY(cudaMemcpyAsync(&got, boff + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    check_scratch(sc, st, "list filter");  // synchronises
    dfree(counts, st);
    dfree(boff, st);
    if (got != expect) throw Error{SLG_EINTERNAL, "list filter: pair count differs from the count"};
}

int64_t run_filter_room(const int32_t* I, const int32_t* J, const int32_t* O, int64_t n, int32_t s,
                        int32_t* I2, int32_t* J2, int32_t* O2, int64_t room, cudaStream_t st) {
    if (n <= 0) return 0;
    const int64_t nb = (n + FT_N - 1) / FT_N;
    int32_t* counts = dalloc<int32_t>((size_t)nb, st);
    int64_t* boff = dalloc<int64_t>((size_t)nb + 1, st);
    k_filter_count<<<(unsigned)nb, FT_THREADS, 0, st>>>(O, n, s, counts);
    SLG_LAUNCH_CHECK();
    scan_i32_to_i64(counts, boff, nb, st);
    int64_t got = 0;
    SLG_CUDA_TRY(cudaMemcpyAsync(&got, boff + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    if (I2 && got <= room) {
        int32_t* sc = new_scratch(st);
        k_filter_write<<<(unsigned)nb, FT_THREADS, 0, st>>>(I, J, O, n, s, boff, I2, J2, O2, got,
                                                            sc + NMODES);
        SLG_LAUNCH_CHECK();
        check_scratch(sc, st, "list filter");  // synchronises
    }
    dfree(counts, st);
    dfree(boff, st);
    return got;
}

void run_count_ensemble(const GraphDev& g, const Plan& p, ModeTimer* mt, cudaStream_t st) {
    const int32_t k = p.ens.k;
    const int64_t ni = p.nitems;
    int32_t* sc = new_scratch(st, NMODES * k);
    int32_t* err = sc + NMODES * k;
    EnsArgs ea = ens_args(p);
    ea.icnt = p.ens.icnt;
    ea.stride = ni;
    // sparse-accumulator and hub-pair rows, up to four lists: every list in one
    // walk (their counting kernels take the thresholds from device memory)
    constexpr unsigned ONE_WALK = (1u << MODE_SPARSE) | (1u << MODE_HUBPAIR);
    unsigned per_list = ENS_PER_LIST;
    EnsArgs* ea_dev = nullptr;
    if (k <= 4) {
        ea_dev = dalloc<EnsArgs>(1, st);
        SLG_CUDA_TRY(cudaMemcpyAsync(ea_dev, &ea, sizeof(EnsArgs), cudaMemcpyHostToDevice, st));
        launch_items<false>(g, p, p.rs_for(p.ens.s[0]), 0, (int32_t)ni, nullptr, nullptr, nullptr,
                            nullptr, nullptr, 0, sc, err, mt, st, ONE_WALK, nullptr, StageArgs{},
                            ea_dev);
        per_list &= ~ONE_WALK;
    }
    // table (and otherwise sparse) handlers: one launch per threshold
    for (int32_t t = 0; t < k; ++t)
        launch_items<false>(g, p, p.rs_for(p.ens.s[t]), 0, (int32_t)ni, p.ens.icnt + t * ni,
                            nullptr, nullptr, nullptr, nullptr, 0, sc + NMODES * t, err, mt, st,
                            per_list);
    // dense handlers: every threshold in one launch
    launch_items<false>(g, p, p.rs_for(p.ens.s[0]), 0, (int32_t)ni, nullptr, nullptr, nullptr,
                        nullptr, nullptr, 0, sc, err, mt, st, ENS_FUSED, &ea);
    check_scratch(sc, st, "ensemble counting pass", NMODES * k);
    dfree(ea_dev, st);
}

void run_digest(RowS rs, const int64_t* rowoff, int32_t r0, int32_t r1, const int32_t* I,
                const int32_t* J, const int32_t* O, int64_t P, unsigned long long* total_dev,
                unsigned long long* rows_dev, cudaStream_t st) {
    if (P <= 0) return;
    int64_t base = 0;
    SLG_CUDA_TRY(cudaMemcpyAsync(&base, rowoff + r0, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    int32_t* sc = new_scratch(st);
    int64_t blocks = (P + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    k_digest<<<(int)blocks, 256, 0, st>>>(I, J, O, P, base, rowoff, r0, r1, rs, total_dev,
                                          rows_dev, sc + NMODES);
    SLG_LAUNCH_CHECK();
    check_scratch(sc, st, "digest");
}

}  // namespace slg
