// The sparse-accumulator handler (MODE_SPARSE) of the counting and fill
// passes: the inner loop of Algorithm 2 (Section III-C) for rows whose
// partners are spread thinly over a wide id range.
#include "kernel_util.cuh"
#include "plan.cuh"

namespace slg {
namespace {

// ========================================================== MODE_SPARSE
//
// Rows whose partners are spread thinly over a wide id range (wedges through
// many high-degree vertices, density far below the dense handlers' bar): a
// sparse accumulator per CTA. One item is a j slice of one row; it is walked
// in tiles of 65536 ids. Per tile:
//   1. every wedge of the tile adds 1 to the 8-bit counter of its partner
//      (|e_i| <= 255 bounds every count); the first increment of a counter
//      appends it to a list of touched counters. Wedge ranges are walked 128
//      entries at a time (four loads in flight per lane); a range expected to
//      hold many entries per tile is split into up to 16 pieces that take
//      every 16th (or P-th) 128-entry chunk, so one heavy range keeps many
//      warps busy instead of one;
//   2. survivors (count >= s) are read off the touched list only (or off the
//      whole tile when more than SP_TOUCH counters were touched), and each
//      counter is cleared as it is read;
//   3. the fill ranks each survivor by the survivors at lower ids (a bitmap
//      of the tile and its per-word prefix), so no sort is needed.
// The counting pass needs two CTA barriers per tile. Hub vertices are counted
// like any other here: a partner may share only hubs with e_i, and only a walk
// over its wedges finds it in a sparse row.

constexpr int SP_WARPS = SP_THREADS / 32;
constexpr int SP_WORDS = SP_TILE / 4;   // four 8-bit counters per word
constexpr int SP_BITS = SP_TILE / 32;   // survivor bitmap words
constexpr int SP_MAXR = 256;            // wedge ranges of a row (|e_i| <= 255)
constexpr int SP_UNROLL = 4;            // 32-entry chunks of a range loaded together
constexpr int SP_CHUNK = 32 * SP_UNROLL;
constexpr int SP_MAXP = 16;             // pieces of one range
constexpr int SP_SLOTS = 1024;          // (range, piece) pairs of an item
constexpr int SP_PIECE = 256;           // expected entries per tile for each piece
static_assert(SP_MAX_SIZE < 256 && SP_MAXR > SP_MAX_SIZE, "8-bit counters");
static_assert(SP_TILE <= 65536, "touched counters are listed as 16-bit offsets");
static_assert(SP_BITS == 4 * SP_THREADS, "bitmap prefix: four words per thread");
static_assert(SP_MAXR <= 256 && SP_MAXP <= 16, "a slot packs a range (8 bits) and a piece (4)");
constexpr size_t sp_smem(bool fill) {
    return sizeof(uint32_t) * SP_WORDS + sizeof(uint16_t) * SP_TOUCH +
           sizeof(int32_t) * 4 * SP_MAXR + sizeof(uint16_t) * SP_SLOTS +
           (fill ? sizeof(uint32_t) * 2 * SP_BITS : 0);
}

template <bool FILL>
__global__ void __launch_bounds__(SP_THREADS, 2)
k_sparse_items(const Item* __restrict__ items, const int32_t* __restrict__ list,
               const int32_t* __restrict__ rank, int32_t item_lo, int32_t item_hi,
               const int32_t* __restrict__ off, const int32_t* __restrict__ wbeg,
               const int32_t* __restrict__ wend, const int32_t* __restrict__ idxTs, RowS rs,
               int32_t* __restrict__ icnt, const int64_t* __restrict__ ioff,
               int32_t* __restrict__ I, int32_t* __restrict__ J, int32_t* __restrict__ O,
               int32_t* __restrict__ queue, int64_t limit, int32_t* __restrict__ err) {
    extern __shared__ __align__(16) uint32_t dyn[];
    uint32_t* ctr = dyn;                                                   // SP_WORDS
    uint16_t* touched = reinterpret_cast<uint16_t*>(ctr + SP_WORDS);      // SP_TOUCH
    int32_t* cur = reinterpret_cast<int32_t*>(touched + SP_TOUCH);        // SP_MAXR
    int32_t* endp = cur + SP_MAXR;                                         // SP_MAXR
    int32_t* adv = endp + SP_MAXR;     // entries of range k taken this tile
    int32_t* npc = adv + SP_MAXR;      // pieces of range k
    uint16_t* slots = reinterpret_cast<uint16_t*>(npc + SP_MAXR);         // SP_SLOTS
    uint32_t* bm = reinterpret_cast<uint32_t*>(slots + SP_SLOTS);         // fill: SP_BITS
    uint32_t* wpre = bm + SP_BITS;                                         // fill: SP_BITS
    __shared__ int32_t tmp[SP_WARPS + 1];
    __shared__ int32_t sh_pos, sh_n;
    __shared__ int32_t sh_nt[2];  // touched counters of the tile, by tile parity
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int32_t lo = rank[item_lo], hi = rank[item_hi];
    // the counters (and the fill's bitmap) start at zero; every tile leaves them so
    for (int32_t w = tid; w < SP_WORDS; w += SP_THREADS) ctr[w] = 0;
    if (FILL)
        for (int32_t w = tid; w < SP_BITS; w += SP_THREADS) bm[w] = 0;

    for (;;) {
        if (tid == 0) {
            sh_pos = lo + atomicAdd(queue, 1);
            sh_n = 0;
            sh_nt[0] = sh_nt[1] = 0;
        }
        __syncthreads();
        const int32_t pos = sh_pos;
        if (pos >= hi) break;
        const int32_t q = list[pos];
        if (FILL && ioff[q + 1] == ioff[q]) {  // nothing to write (same in every thread)
            __syncthreads();
            continue;
        }
        const Item it = items[q];
        const int32_t i = it.row;
        const int32_t s = rs.s_of(i);
        const int32_t ib = rs.base_of(i);
        const int32_t e0 = off[i];
        const int32_t ne = off[i + 1] - e0;
        // wedge ranges of the row, cursors at the item's first partner
        for (int32_t k = tid; k < ne; k += SP_THREADS) {
            const int32_t e = e0 + k;
            const int32_t b0 = wbeg[e], t = wend[e];
            if (t > b0) {
                const int32_t c = (__ldg(&idxTs[b0]) >= it.jlo)
                                      ? b0 : lower_bound_dev(idxTs, b0, t, it.jlo);
                if (c < t) {
                    const int32_t slot = atomicAdd(&sh_n, 1);
                    if (slot < SP_MAXR) {
                        cur[slot] = c;
                        endp[slot] = t;
                    } else {
                        atomicOr(err, ERR_TABLE);  // binning admits |e_i| <= 255 only
                    }
                }
            }
        }
        const int64_t obase = FILL ? ioff[q] - ioff[item_lo] : 0;
        int64_t out_pos = 0;   // fill: the item's pairs before the tile (same in every thread)
        int32_t my_count = 0;  // counting pass: this thread's survivors so far
        __syncthreads();
        const int32_t nr = min(sh_n, SP_MAXR);
        // pieces per range, from its density: entries per id times the tile width
        int32_t np = 0;
        if (tid < nr) {
            const int32_t c = cur[tid], e = endp[tid];
            const int64_t idspan = (int64_t)__ldg(&idxTs[e - 1]) - __ldg(&idxTs[c]) + 1;
            const int64_t expect = (int64_t)(e - c) * SP_TILE / idspan;
            np = (int32_t)min((int64_t)SP_MAXP, max((int64_t)1, (expect + SP_PIECE - 1) / SP_PIECE));
            adv[tid] = 0;
        }
        int32_t nslots = 0;
        int32_t first = block_excl_scan<SP_THREADS>(np, &nslots, tmp);
        if (nslots > SP_SLOTS) {  // too many: one piece per range
            np = tid < nr ? 1 : 0;
            first = tid;
            nslots = nr;
        }
        if (tid < nr) {
            npc[tid] = np;
            for (int32_t u = 0; u < np; ++u) slots[first + u] = (uint16_t)((tid << 4) | u);
        }
        __syncthreads();
        int par = 0;
        for (int32_t t0 = it.jlo; t0 < it.jhi; t0 += SP_TILE, par ^= 1) {
            const int32_t t1 = min(t0 + SP_TILE, it.jhi);
            const int32_t span = t1 - t0;
            // 1. wedges of the tile: a warp takes (range, piece) slots; piece u of
            // a range split P ways walks chunks u, u+P, u+2P, ... from the
            // range's cursor and stops at its first chunk that is not entirely
            // inside the tile (every later chunk lies beyond the tile)
            for (int32_t qs = warp; qs < nslots; qs += SP_WARPS) {
                const int32_t sl = slots[qs];
                const int32_t k = sl >> 4, piece = sl & 15;
                const int32_t P = npc[k];
                const int32_t c0 = cur[k];
                const int32_t e = endp[k];
                int32_t taken = 0;
                for (int32_t base = c0 + piece * SP_CHUNK; base < e; base += P * SP_CHUNK) {
                    int32_t jv[SP_UNROLL];
#pragma unroll
                    for (int u = 0; u < SP_UNROLL; ++u) {
                        const int32_t p = base + 32 * u + lane;
                        jv[u] = p < e ? __ldg(&idxTs[p]) : INT32_MAX;
                    }
                    int n = 0;
#pragma unroll
                    for (int u = 0; u < SP_UNROLL; ++u) {
                        const bool valid = jv[u] < t1;
                        bool first_touch = false;
                        int32_t slot = 0;
                        if (valid) {
                            slot = jv[u] - t0;
                            const int sh = (slot & 3) << 3;
                            const uint32_t old = atomicAdd(&ctr[slot >> 2], 1u << sh);
                            first_touch = ((old >> sh) & 0xffu) == 0;
                        }
                        const unsigned fb = __ballot_sync(0xffffffffu, first_touch);
                        if (fb) {
                            int32_t b = 0;
                            if (lane == 0) b = atomicAdd(&sh_nt[par], __popc(fb));
                            b = __shfl_sync(0xffffffffu, b, 0);
                            const int32_t at = b + __popc(fb & lt);
                            if (first_touch && at < SP_TOUCH) touched[at] = (uint16_t)slot;
                        }
                        n += __popc(__ballot_sync(0xffffffffu, valid));
                    }
                    taken += n;
                    if (n < SP_CHUNK) break;
                }
                if (lane == 0 && taken) atomicAdd(&adv[k], taken);
            }
            __syncthreads();
            if (tid < nr) {  // advance each range past the entries this tile took
                cur[tid] += adv[tid];
                adv[tid] = 0;
            }
            const int32_t nt = sh_nt[par];
            if (tid == 0) sh_nt[par ^ 1] = 0;  // for the next tile (last read a tile ago)
            const bool listed = nt <= SP_TOUCH;
            const int32_t nwords = (span + 3) >> 2;
            if (!FILL) {
                // 2. survivors, clearing each counter as it is read
                if (listed) {
                    for (int32_t x = tid; x < nt; x += SP_THREADS) {
                        const int32_t slot = touched[x];
                        const int sh = (slot & 3) << 3;
                        const uint32_t old = atomicAnd(&ctr[slot >> 2], ~(0xffu << sh));
                        my_count += ((int32_t)((old >> sh) & 0xffu) >= s) ? 1 : 0;
                    }
                } else {
                    for (int32_t w = tid; w < nwords; w += SP_THREADS) {
                        const uint32_t v = ctr[w];
                        if (!v) continue;
                        ctr[w] = 0;
#pragma unroll
                        for (int r = 0; r < 4; ++r)
                            my_count += ((int32_t)((v >> (8 * r)) & 0xffu) >= s) ? 1 : 0;
                    }
                }
                __syncthreads();  // the touched list is refilled by the next tile
                continue;
            }
            // 2. survivors into the bitmap
            int32_t mine = 0;
            if (listed) {
                for (int32_t x = tid; x < nt; x += SP_THREADS) {
                    const int32_t slot = touched[x];
                    const int32_t c = (int32_t)((ctr[slot >> 2] >> ((slot & 3) << 3)) & 0xffu);
                    if (c >= s) {
                        ++mine;
                        atomicOr(&bm[slot >> 5], 1u << (slot & 31));
                    }
                }
            } else {
                for (int32_t w = tid; w < nwords; w += SP_THREADS) {
                    const uint32_t v = ctr[w];
                    if (!v) continue;
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int32_t slot = 4 * w + r;
                        if (slot < span && (int32_t)((v >> (8 * r)) & 0xffu) >= s) {
                            ++mine;
                            atomicOr(&bm[slot >> 5], 1u << (slot & 31));
                        }
                    }
                }
            }
            // 3. rank of a survivor: survivors in earlier bitmap words plus
            // earlier bits of its own word (the scan's barriers order the
            // bitmap writes above before these reads)
            uint32_t wv[4];
            int32_t sum = 0;
            __syncthreads();
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                wv[r] = bm[4 * tid + r];
                sum += __popc(wv[r]);
            }
            int32_t tile_total = 0;
            int32_t acc = block_excl_scan<SP_THREADS>(sum, &tile_total, tmp);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                wpre[4 * tid + r] = (uint32_t)acc;
                acc += __popc(wv[r]);
            }
            __syncthreads();
            const int64_t base = obase + out_pos;
            auto emit = [&](int32_t slot, int32_t c) {
                const uint32_t wb = bm[slot >> 5];
                const int64_t p2 = base + wpre[slot >> 5] + __popc(wb & ((1u << (slot & 31)) - 1u));
                if (p2 < limit) {
                    I[p2] = i - ib;
                    J[p2] = t0 + slot - ib;
                    O[p2] = c;
                } else {
                    atomicOr(err, ERR_BOUNDS);
                }
            };
            // survivors are written and every counter of the tile is cleared
            if (listed) {
                for (int32_t x = tid; x < nt; x += SP_THREADS) {
                    const int32_t slot = touched[x];
                    const int sh = (slot & 3) << 3;
                    const uint32_t old = atomicAnd(&ctr[slot >> 2], ~(0xffu << sh));
                    const int32_t c = (int32_t)((old >> sh) & 0xffu);
                    if (c >= s) emit(slot, c);
                }
            } else {
                for (int32_t w = tid; w < nwords; w += SP_THREADS) {
                    const uint32_t v = ctr[w];
                    if (!v) continue;
                    ctr[w] = 0;
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int32_t slot = 4 * w + r;
                        const int32_t c = (int32_t)((v >> (8 * r)) & 0xffu);
                        if (slot < span && c >= s) emit(slot, c);
                    }
                }
            }
            out_pos += tile_total;
            __syncthreads();  // bitmap reads done; the touched list is refilled next tile
            if (tile_total > 0)
                for (int32_t w = tid; w < SP_BITS; w += SP_THREADS) bm[w] = 0;
            // (the next tile's bitmap writes follow its first barrier)
        }
        if (!FILL) {
            int32_t total = 0;
            block_excl_scan<SP_THREADS>(my_count, &total, tmp);
            if (tid == 0) icnt[q] = total;
        }
        __syncthreads();
    }
}

// ========================================================= MODE_WSPARSE
//
// The sparse accumulator at warp granularity, for sparse rows with at most 32
// vertices (one wedge range per lane): a warp owns an item and a private tile
// of 4096 8-bit counters, so many tiles are in flight per SM and no CTA barrier
// is ever taken. Per tile (which starts at the smallest next partner of any
// range, so empty stretches of the id range cost nothing):
//   1. ranges with a partner inside the tile load 32 entries each, four
//      ranges per round, and count them; a counter's first increment appends
//      it to the warp's touched list;
//   2. survivors are read off the touched list (or the whole tile when it
//      overflows); the counting pass adds them up, the fill marks them in a
//      bitmap of the tile;
//   3. fill: the bitmap is walked in id order, four partners per lane, and
//      survivors go through a ring to 128-byte-aligned chunk stores, as in the
//      warp dense handler;
//   4. the touched counters are cleared.

constexpr int WS_WARPS = 16;
constexpr int WS_TILE = 4096;
constexpr int WS_WORDS = WS_TILE / 4;   // four 8-bit counters per word
constexpr int WS_BITS = WS_TILE / 32;   // survivor bitmap words (fill)
constexpr int WS_TOUCH = 256;           // touched counters listed per tile
constexpr int WS_RING = 256;            // fill: survivors waiting for an aligned store
constexpr int WS_GROUP = 4;             // ranges loaded together per round
static_assert(WS_BITS == 4 * 32, "the bitmap walk takes four partners per lane and round");
static_assert(WS_MAXE <= 32 && WS_MAXE < 256, "one range per lane; 8-bit counts");
// fill: the ring keeps ids (32 bits) and counts (8 bits) in separate arrays
constexpr size_t ws_warp_words(bool fill) {
    return WS_WORDS + WS_TOUCH / 2 + (fill ? WS_BITS + WS_RING + WS_RING / 4 : 0);
}
constexpr size_t ws_smem(bool fill) { return sizeof(uint32_t) * ws_warp_words(fill) * WS_WARPS; }

template <bool FILL>
__global__ void __launch_bounds__(WS_WARPS * 32, FILL ? 2 : 3)
k_wsparse_items(const Item* __restrict__ items, const int32_t* __restrict__ list,
                const int32_t* __restrict__ rank, int32_t item_lo, int32_t item_hi,
                const int32_t* __restrict__ off, const int32_t* __restrict__ wbeg,
                const int32_t* __restrict__ wend, const int32_t* __restrict__ idxTs, RowS rs,
                int32_t* __restrict__ icnt, const int64_t* __restrict__ ioff,
                int32_t* __restrict__ I, int32_t* __restrict__ J, int32_t* __restrict__ O,
                int32_t* __restrict__ queue, int64_t limit, int32_t* __restrict__ err) {
    extern __shared__ __align__(16) uint32_t dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* ctr = dyn + (size_t)warp * ws_warp_words(FILL);           // WS_WORDS
    uint16_t* touched = reinterpret_cast<uint16_t*>(ctr + WS_WORDS);    // WS_TOUCH
    uint32_t* bm = reinterpret_cast<uint32_t*>(touched + WS_TOUCH);     // fill: WS_BITS
    int32_t* ring_j = reinterpret_cast<int32_t*>(bm + WS_BITS);          // fill: WS_RING
    uint8_t* ring_o = reinterpret_cast<uint8_t*>(ring_j + WS_RING);      // fill: WS_RING
    const unsigned lt = (1u << lane) - 1u;
    const int32_t lo = rank[item_lo], hi = rank[item_hi];
    for (int32_t w = lane; w < WS_WORDS; w += 32) ctr[w] = 0;
    if (FILL)
        for (int32_t w = lane; w < WS_BITS; w += 32) bm[w] = 0;
    __syncwarp();

    for (;;) {
        int32_t pos = 0;
        if (lane == 0) pos = lo + atomicAdd(queue, 1);
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (pos >= hi) break;
        const int32_t q = list[pos];
        if (FILL && ioff[q + 1] == ioff[q]) continue;  // nothing to write
        const Item it = items[q];
        const int32_t i = it.row;
        const int32_t s = rs.s_of(i);
        const int32_t ib = rs.base_of(i);
        const int32_t e0 = off[i];
        const int32_t ne = off[i + 1] - e0;
        if (ne > 32 && lane == 0) atomicOr(err, ERR_TABLE);  // binning admits |e_i| <= 32
        // lane k holds the wedge range of the row's k-th vertex, cursor at jlo
        int32_t cur = 0, end = 0, nxt = INT32_MAX;
        if (lane < ne) {
            const int32_t e = e0 + lane;
            const int32_t b0 = wbeg[e], t = wend[e];
            if (t > b0) {
                const int32_t c = (__ldg(&idxTs[b0]) >= it.jlo)
                                      ? b0 : lower_bound_dev(idxTs, b0, t, it.jlo);
                if (c < t) {
                    cur = c;
                    end = t;
                    nxt = __ldg(&idxTs[c]);
                }
            }
        }
        int64_t wpos = FILL ? ioff[q] - ioff[item_lo] : 0;  // next output position
        int32_t rhead = 0, rcount = 0;
        int32_t need = FILL ? 32 - (int32_t)((reinterpret_cast<uintptr_t>(I + wpos) >> 2) & 31) : 32;
        int32_t my_count = 0;
        for (;;) {
            const int32_t t0 = __reduce_min_sync(0xffffffffu, nxt);  // next partner of any range
            if (t0 >= it.jhi) break;
            const int32_t t1 = min(t0 + WS_TILE, it.jhi);
            const int32_t span = t1 - t0;
            // 1. wedges of the tile
            unsigned act = __ballot_sync(0xffffffffu, nxt < t1);
            int32_t nt = 0;  // counters touched (same in every lane)
            while (act) {
                int32_t kk[WS_GROUP], vv[WS_GROUP];
                unsigned aa = act;
#pragma unroll
                for (int g = 0; g < WS_GROUP; ++g) {
                    int32_t k = -1;
                    if (aa) {
                        k = __ffs(aa) - 1;
                        aa &= aa - 1u;
                    }
                    kk[g] = k;
                    const int32_t c = __shfl_sync(0xffffffffu, cur, k & 31);
                    const int32_t e = __shfl_sync(0xffffffffu, end, k & 31);
                    const int32_t p = c + lane;
                    vv[g] = (k >= 0 && p < e) ? __ldg(&idxTs[p]) : INT32_MAX;
                }
#pragma unroll
                for (int g = 0; g < WS_GROUP; ++g) {
                    const int32_t k = kk[g];
                    if (k < 0) break;
                    const bool valid = vv[g] < t1;
                    bool first = false;
                    int32_t slot = 0;
                    if (valid) {
                        slot = vv[g] - t0;
                        const int sh = (slot & 3) << 3;
                        const uint32_t old = atomicAdd(&ctr[slot >> 2], 1u << sh);
                        first = ((old >> sh) & 0xffu) == 0;
                    }
                    const unsigned fb = __ballot_sync(0xffffffffu, first);
                    if (fb) {
                        const int32_t at = nt + __popc(fb & lt);
                        if (first && at < WS_TOUCH) touched[at] = (uint16_t)slot;
                        nt += __popc(fb);
                    }
                    const int n = __popc(__ballot_sync(0xffffffffu, valid));
                    // the first entry not taken is the range's next partner
                    const int32_t nx = __shfl_sync(0xffffffffu, vv[g], n & 31);
                    if (lane == k) {
                        cur += n;
                        if (n < 32) nxt = nx;
                    }
                    if (n < 32) act &= ~(1u << k);
                }
            }
            __syncwarp();
            const bool listed = nt <= WS_TOUCH;
            const int32_t nwords = (span + 3) >> 2;
            // 2. survivors
            if (listed) {
                for (int32_t x = lane; x < nt; x += 32) {
                    const int32_t slot = touched[x];
                    const int32_t c = (int32_t)((ctr[slot >> 2] >> ((slot & 3) << 3)) & 0xffu);
                    if (c >= s) {
                        if (FILL)
                            atomicOr(&bm[slot >> 5], 1u << (slot & 31));
                        else
                            ++my_count;
                    }
                }
            } else {
                for (int32_t w = lane; w < nwords; w += 32) {
                    const uint32_t v = ctr[w];
                    if (!v) continue;
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int32_t slot = 4 * w + r;
                        if (slot < span && (int32_t)((v >> (8 * r)) & 0xffu) >= s) {
                            if (FILL)
                                atomicOr(&bm[slot >> 5], 1u << (slot & 31));
                            else
                                ++my_count;
                        }
                    }
                }
            }
            __syncwarp();
            if (FILL) {
                // 3. survivors in id order: round r covers partners 128r .. 128r+127,
                // lane l the four partners 128r + 4l .. 128r + 4l + 3 (one counter word);
                // only rounds whose four bitmap words hold a survivor are visited
                const uint32_t b4 = bm[4 * lane] | bm[4 * lane + 1] | bm[4 * lane + 2] | bm[4 * lane + 3];
                for (unsigned rounds = __ballot_sync(0xffffffffu, b4 != 0); rounds;
                     rounds &= rounds - 1u) {
                    const int32_t r = __ffs(rounds) - 1;
                    const uint32_t nib = (bm[4 * r + (lane >> 3)] >> ((lane & 7) * 4)) & 0xfu;
                    const uint32_t cw = nib ? ctr[32 * r + lane] : 0u;
                    const int32_t mine = __popc(nib);
                    int32_t inc = mine;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const int32_t y = __shfl_up_sync(0xffffffffu, inc, d);
                        if (lane >= d) inc += y;
                    }
                    const int32_t tot = __shfl_sync(0xffffffffu, inc, 31);
                    int32_t slot = rhead + rcount + inc - mine;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        if ((nib >> b) & 1u) {
                            ring_j[slot & (WS_RING - 1)] = t0 + 128 * r + 4 * lane + b;
                            ring_o[slot & (WS_RING - 1)] = (uint8_t)((cw >> (8 * b)) & 0xffu);
                            ++slot;
                        }
                    }
                    rcount += tot;
                    __syncwarp();
                    while (rcount >= need) {
                        if (lane < need) {
                            const int32_t x = (rhead + lane) & (WS_RING - 1);
                            const int64_t p2 = wpos + lane;
                            if (p2 < limit) {
                                I[p2] = i - ib;
                                J[p2] = ring_j[x] - ib;
                                O[p2] = ring_o[x];
                            } else {
                                atomicOr(err, ERR_BOUNDS);
                            }
                        }
                        rhead = (rhead + need) & (WS_RING - 1);
                        rcount -= need;
                        wpos += need;
                        need = 32;
                    }
                    __syncwarp();
                }
                if (b4) {  // clear this lane's four words
                    bm[4 * lane] = 0;
                    bm[4 * lane + 1] = 0;
                    bm[4 * lane + 2] = 0;
                    bm[4 * lane + 3] = 0;
                }
            }
            // 4. clear what the tile used (every read above is done)
            if (listed) {
                for (int32_t x = lane; x < nt; x += 32) ctr[touched[x] >> 2] = 0;
            } else {
                for (int32_t w = lane; w < nwords; w += 32) ctr[w] = 0;
            }
            __syncwarp();
        }
        if (FILL && rcount > 0) {  // the item's last, partial chunk
            if (lane < rcount) {
                const int32_t x = (rhead + lane) & (WS_RING - 1);
                const int64_t p2 = wpos + lane;
                if (p2 < limit) {
                    I[p2] = i - ib;
                    J[p2] = ring_j[x] - ib;
                    O[p2] = ring_o[x];
                } else {
                    atomicOr(err, ERR_BOUNDS);
                }
            }
            __syncwarp();
        }
        if (!FILL) {
            const int32_t total = (int32_t)__reduce_add_sync(0xffffffffu, (unsigned)my_count);
            if (lane == 0) icnt[q] = total;
        }
    }
}

}  // namespace

void sparse_setup(int sms, int ctas[2]) {
    for (int f = 0; f < 2; ++f) {
        const size_t smem = sp_smem(f == 1);
        auto kern = f ? k_sparse_items<true> : k_sparse_items<false>;
        SLG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        int d = 0;
        SLG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, kern, SP_THREADS, smem));
        ctas[f] = sms * (d > 0 ? d : 1);
    }
}

void wsparse_setup(int sms, int ctas[2]) {
    for (int f = 0; f < 2; ++f) {
        const size_t smem = ws_smem(f == 1);
        auto kern = f ? k_wsparse_items<true> : k_wsparse_items<false>;
        SLG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        int d = 0;
        SLG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, kern, WS_WARPS * 32, smem));
        ctas[f] = sms * (d > 0 ? d : 1);
    }
}

void launch_wsparse(bool fill, int ctas, const GraphDev& g, const Plan& p, RowS rs,
                    int32_t item_lo, int32_t item_hi, int32_t* icnt, const int64_t* ioff,
                    int32_t* I, int32_t* J, int32_t* O, int32_t* queue, int64_t limit,
                    int32_t* err, cudaStream_t st) {
    if (fill)
        k_wsparse_items<true><<<ctas, WS_WARPS * 32, ws_smem(true), st>>>(
            p.items, p.mode_list[MODE_WSPARSE], p.mode_rank[MODE_WSPARSE], item_lo, item_hi,
            g.off, p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I, J, O, queue, limit, err);
    else
        k_wsparse_items<false><<<ctas, WS_WARPS * 32, ws_smem(false), st>>>(
            p.items, p.mode_list[MODE_WSPARSE], p.mode_rank[MODE_WSPARSE], item_lo, item_hi,
            g.off, p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I, J, O, queue, limit, err);
    SLG_LAUNCH_CHECK();
}

void launch_sparse(bool fill, int ctas, const GraphDev& g, const Plan& p, RowS rs,
                   int32_t item_lo, int32_t item_hi, int32_t* icnt, const int64_t* ioff,
                   int32_t* I, int32_t* J, int32_t* O, int32_t* queue, int64_t limit,
                   int32_t* err, cudaStream_t st) {
    if (fill)
        k_sparse_items<true><<<ctas, SP_THREADS, sp_smem(true), st>>>(
            p.items, p.mode_list[MODE_SPARSE], p.mode_rank[MODE_SPARSE], item_lo, item_hi, g.off,
            p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I, J, O, queue, limit, err);
    else
        k_sparse_items<false><<<ctas, SP_THREADS, sp_smem(false), st>>>(
            p.items, p.mode_list[MODE_SPARSE], p.mode_rank[MODE_SPARSE], item_lo, item_hi, g.off,
            p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I, J, O, queue, limit, err);
    SLG_LAUNCH_CHECK();
}

}  // namespace slg
