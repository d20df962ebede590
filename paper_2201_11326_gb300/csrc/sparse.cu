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

// ENS4: the counting pass of an ensemble of at most four lists (*eap, in device
// memory): every list counted in the one walk.
template <bool FILL, bool ENS4 = false>
__global__ void __launch_bounds__(SP_THREADS, 2)
k_sparse_items(const Item* __restrict__ items, const int32_t* __restrict__ list,
               const int32_t* __restrict__ rank, int32_t item_lo, int32_t item_hi,
               const int32_t* __restrict__ off, const int32_t* __restrict__ wbeg,
               const int32_t* __restrict__ wend, const int32_t* __restrict__ idxTs, RowS rs,
               int32_t* __restrict__ icnt, const int64_t* __restrict__ ioff,
               int32_t* __restrict__ I, int32_t* __restrict__ J, int32_t* __restrict__ O,
               int32_t* __restrict__ queue, int64_t limit, int32_t* __restrict__ err,
               StageArgs sa, const EnsArgs* __restrict__ eap) {
    static_assert(!(FILL && ENS4), "an ensemble's lists are counted here, filled one at a time");
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
    __shared__ long long sh_cpos, sh_cend;  // staging: the CTA's chunk of the pool
    __shared__ int32_t sh_sovf;             // staging: the item's pairs did not fit
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool stg = FILL && sa.J != nullptr;  // the counting pass, staging pairs
    const unsigned lt = (1u << lane) - 1u;
    const int32_t lo = rank[item_lo], hi = rank[item_hi];
    // the counters (and the fill's bitmap) start at zero; every tile leaves them so
    for (int32_t w = tid; w < SP_WORDS; w += SP_THREADS) ctr[w] = 0;
    if (FILL)
        for (int32_t w = tid; w < SP_BITS; w += SP_THREADS) bm[w] = 0;

    if (tid == 0) sh_cpos = sh_cend = 0;
    for (;;) {
        if (tid == 0) {
            sh_n = 0;
            sh_nt[0] = sh_nt[1] = 0;
            sh_sovf = 0;
            bool room = true;
            if (stg && sh_cend - sh_cpos < sa.min_room) {  // a fresh chunk, if the pool has one
                const unsigned long long c = atomicAdd(sa.cursor, (unsigned long long)sa.chunk);
                room = (int64_t)c + sa.chunk <= sa.cap;
                if (room) {
                    sh_cpos = (long long)c;
                    sh_cend = (long long)c + sa.chunk;
                }
            }
            // a spent pool ends the staging launch; the counting kernel takes the
            // items from this queue position on
            sh_pos = room ? lo + atomicAdd(queue, 1) : hi;
        }
        __syncthreads();
        const int32_t pos = sh_pos;
        if (pos >= hi) break;
        const int32_t q = list[pos];
        if (FILL && !stg && (ioff[q + 1] == ioff[q] || (sa.at && sa.at[q] >= 0))) {
            __syncthreads();  // nothing to write, or staged (same in every thread)
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
        const int64_t obase = !FILL ? 0 : stg ? (int64_t)sh_cpos : ioff[q] - ioff[item_lo];
        const int64_t olimit = stg ? (int64_t)sh_cend : limit;
        int64_t out_pos = 0;   // fill: the item's pairs before the tile (same in every thread)
        int32_t my_count = 0;  // counting pass: this thread's survivors so far
        // ENS4: this thread's survivors of each list so far, and the thresholds
        // (a list beyond the ensemble never counts)
        int32_t en0 = 0, en1 = 0, en2 = 0, en3 = 0;
        const int32_t es0 = ENS4 ? eap->s[0] : 0;
        const int32_t es1 = ENS4 && eap->k > 1 ? eap->s[1] : INT32_MAX;
        const int32_t es2 = ENS4 && eap->k > 2 ? eap->s[2] : INT32_MAX;
        const int32_t es3 = ENS4 && eap->k > 3 ? eap->s[3] : INT32_MAX;
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
                        const int32_t c = (int32_t)((old >> sh) & 0xffu);
                        if (ENS4) {
                            en0 += c >= es0 ? 1 : 0;
                            en1 += c >= es1 ? 1 : 0;
                            en2 += c >= es2 ? 1 : 0;
                            en3 += c >= es3 ? 1 : 0;
                        } else {
                            my_count += c >= s ? 1 : 0;
                        }
                    }
                } else {
                    for (int32_t w = tid; w < nwords; w += SP_THREADS) {
                        const uint32_t v = ctr[w];
                        if (!v) continue;
                        ctr[w] = 0;
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const int32_t c = (int32_t)((v >> (8 * r)) & 0xffu);
                            if (ENS4) {
                                en0 += c >= es0 ? 1 : 0;
                                en1 += c >= es1 ? 1 : 0;
                                en2 += c >= es2 ? 1 : 0;
                                en3 += c >= es3 ? 1 : 0;
                            } else {
                                my_count += c >= s ? 1 : 0;
                            }
                        }
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
            if (!__syncthreads_or(mine > 0)) {
                // no survivor: clear the tile's counters, as the counting pass does
                if (listed) {
                    for (int32_t x = tid; x < nt; x += SP_THREADS) {
                        const int32_t slot = touched[x];
                        ctr[slot >> 2] = 0u;
                    }
                } else {
                    for (int32_t w = tid; w < nwords; w += SP_THREADS) ctr[w] = 0u;
                }
                __syncthreads();  // the touched list is refilled by the next tile
                continue;
            }
            // 3. rank of a survivor: survivors in earlier bitmap words plus
            // earlier bits of its own word (the scan's barriers order the
            // bitmap writes above before these reads)
            uint32_t wv[4];
            int32_t sum = 0;
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
                if (p2 < olimit) {
                    if (stg) {
                        sa.J[p2] = t0 + slot - ib;
                        sa.O[p2] = (uint8_t)c;
                    } else {
                        I[p2] = i - ib;
                        J[p2] = t0 + slot - ib;
                        O[p2] = c;
                    }
                } else if (stg) {
                    sh_sovf = 1;  // the item is filled again later
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
        if (!FILL && ENS4) {
            int32_t t0c = 0, t1c = 0, t2c = 0, t3c = 0;
            block_excl_scan<SP_THREADS>(en0, &t0c, tmp);
            block_excl_scan<SP_THREADS>(en1, &t1c, tmp);
            block_excl_scan<SP_THREADS>(en2, &t2c, tmp);
            block_excl_scan<SP_THREADS>(en3, &t3c, tmp);
            if (tid == 0) {
                const int32_t tc[4] = {t0c, t1c, t2c, t3c};
                for (int32_t t = 0; t < eap->k; ++t) eap->icnt[t * eap->stride + q] = tc[t];
            }
        } else if (!FILL) {
            int32_t total = 0;
            block_excl_scan<SP_THREADS>(my_count, &total, tmp);
            if (tid == 0) icnt[q] = total;
        } else if (stg) {
            __syncthreads();  // every write (and overflow flag) of the item is done
            if (tid == 0) {
                icnt[q] = (int32_t)out_pos;
                if (!sh_sovf) {
                    sa.at[q] = obase;
                    sh_cpos = obase + out_pos;
                }
            }
        }
        __syncthreads();
    }
}

// ========================================================= MODE_WSPARSE
//
// Sparse rows with at most 32 vertices (one wedge range per lane) whose
// partners are spread thinly over a wide id range: one warp per item, counting
// in rounds into a private open-addressing hash table, so the on-chip state
// grows with the wedges counted, not with the id span they cover (a
// direct-addressed tile of 8-bit counters holds one id per byte; the table holds
// one partner per 8 bytes at half load, which wins below one wedge per 8 ids).
// A round takes every wedge with partner j in [t0, t1):
//   1. t0 is the smallest next partner over the ranges; from each range's
//      density (entries left per id of its remaining span) a round end t1e is
//      chosen for about HS_TARGET wedges, and each range whose next partner
//      lies below t1e gets a load window of its next L entries (the expected
//      count plus a margin, at least 2; the windows together at most HS_CAP
//      entries in HS_STEPS loads of 32, else t1e shrinks);
//   2. the windows are loaded, eight independent 32-entry loads in flight, into
//      a staging buffer. t1 = the smallest last entry of a window that does not
//      reach its range's end (every entry below it is inside its window), the
//      next partner of a range without a window, or the item's end;
//   3. every staged entry below t1 adds 1 to its partner's count in the table
//      (a 32-bit slot: (j - t0 + 1) << 8 | count, placed by compare-and-swap).
//      Each range advances past its entries below t1; its next partner is the
//      first staged entry it did not take, so a range becomes active again only
//      when a later round's end passes that partner;
//   4. the table is scanned: partners with count >= s are survivors; the
//      counting pass adds them up, the fill sorts them by j (a warp bitonic
//      sort) and writes them in order. The table is cleared as it is read.
// Every round makes progress: a window holds at least two entries unless it
// reaches its range's end, so its last entry exceeds t0, and a range without a
// window has its next partner at or beyond t1e > t0; hence t1 > t0, and the
// next round starts at or beyond t1 (every entry below t1 has been taken).

constexpr int HS_WARPS = 8;              // warps per CTA
constexpr int HS_SLOTS = 1024;           // table slots per warp
constexpr int HS_LOG = 10;
constexpr int HS_CAP = 512;              // entries loaded per round at most (table half full)
constexpr int HS_STEPS = 32;             // 32-entry loads per round at most
constexpr int HS_TARGET = 384;           // wedges aimed at per round
constexpr int32_t HS_SPAN = 1 << 23;     // ids per round at most: keys + 1 fit 24 bits
constexpr int HS_GROUP = 8;              // loads issued together
static_assert((1 << HS_LOG) == HS_SLOTS && 2 * HS_CAP <= HS_SLOTS, "table at most half full");
static_assert(HS_STEPS == 32, "one step per lane in the step table");
static_assert(HS_CAP <= HS_STEPS * 32, "survivors are sorted in the staging buffer");
static_assert(WS_MAXE <= 32 && WS_MAXE < 256, "one range per lane; 8-bit counts");
// per warp: table, staging buffer (also the fill's survivor list), step table
constexpr size_t HS_WARP_WORDS = HS_SLOTS + HS_STEPS * 32 + 2 * HS_STEPS;
constexpr size_t HS_SMEM = sizeof(uint32_t) * HS_WARP_WORDS * HS_WARPS;

// Ascending bitonic sort of n <= HS_CAP packed survivors (key << 8 | count) in
// shared memory by one warp; n <= 32 in registers.
__device__ __forceinline__ void warp_sort_u32(uint32_t* a, int32_t n, int lane) {
    if (n <= 1) return;
    if (n <= 32) {
        uint32_t x = lane < n ? a[lane] : 0xffffffffu;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
                const bool up = (lane & k) == 0, low = (lane & j) == 0;
                x = (low == up) ? min(x, y) : max(x, y);
            }
        }
        __syncwarp();
        if (lane < n) a[lane] = x;
        __syncwarp();
        return;
    }
    int32_t P = 64;
    while (P < n) P <<= 1;
    for (int32_t t = n + lane; t < P; t += 32) a[t] = 0xffffffffu;
    __syncwarp();
    for (int32_t k = 2; k <= P; k <<= 1) {
        for (int32_t j = k >> 1; j > 0; j >>= 1) {
            for (int32_t t = lane; t < P; t += 32) {
                const int32_t u = t ^ j;
                if (u > t) {
                    const uint32_t x = a[t], y = a[u];
                    if ((x > y) == ((t & k) == 0)) {
                        a[t] = y;
                        a[u] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
}

template <bool FILL>
__global__ void __launch_bounds__(HS_WARPS * 32)
k_wsparse_items(const Item* __restrict__ items, const int32_t* __restrict__ list,
                const int32_t* __restrict__ rank, int32_t item_lo, int32_t item_hi,
                const int32_t* __restrict__ off, const int32_t* __restrict__ wbeg,
                const int32_t* __restrict__ wend, const int32_t* __restrict__ idxTs, RowS rs,
                int32_t* __restrict__ icnt, const int64_t* __restrict__ ioff,
                int32_t* __restrict__ I, int32_t* __restrict__ J, int32_t* __restrict__ O,
                int32_t* __restrict__ queue, int64_t limit, int32_t* __restrict__ err) {
    extern __shared__ __align__(16) uint32_t dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u;
    uint32_t* tab = dyn + (size_t)warp * HS_WARP_WORDS;                    // HS_SLOTS
    int32_t* stage = reinterpret_cast<int32_t*>(tab + HS_SLOTS);           // HS_STEPS * 32
    int32_t* st_p0 = stage + HS_STEPS * 32;                                // HS_STEPS
    int32_t* st_meta = st_p0 + HS_STEPS;                                   // HS_STEPS
    const int32_t lo = rank[item_lo], hi = rank[item_hi];
    for (int32_t w = lane; w < HS_SLOTS; w += 32) tab[w] = 0u;
    __syncwarp();

    for (;;) {
        int32_t pos = 0;
        if (lane == 0) pos = lo + atomicAdd(queue, 1);
        pos = __shfl_sync(FULL, pos, 0);
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
        // lane k: the wedge range of the row's k-th vertex, cursor at jlo
        int32_t cur = 0, end = 0, nxt = INT32_MAX, last = 0;
        if (lane < ne) {
            const int32_t e = e0 + lane;
            const int32_t b0 = wbeg[e], t = wend[e];
            if (t > b0) {
                const int32_t c = (__ldg(&idxTs[b0]) >= it.jlo) ? b0
                                                                : lower_bound_dev(idxTs, b0, t, it.jlo);
                if (c < t) {
                    cur = c;
                    end = t;
                    nxt = __ldg(&idxTs[c]);
                    last = __ldg(&idxTs[t - 1]);
                }
            }
        }
        int64_t wpos = FILL ? ioff[q] - ioff[item_lo] : 0;  // next output position
        int32_t my_count = 0;
        for (;;) {
            const int32_t t0 = __reduce_min_sync(FULL, nxt);
            if (t0 >= it.jhi) break;
            // 1. the round's end and each range's load window. A range with n
            // entries left spread over the ids [nxt, last] is expected to hold
            // min(n, (t0 + span - nxt) * n / (last - nxt + 1)) entries below t0 +
            // span; the span is set so that the ranges together expect about
            // HS_TARGET (a few multiplicative corrections of a first estimate)
            const bool live = nxt < it.jhi;
            const float left = (float)(end - cur);
            const float dens = live ? left / ((float)last - (float)nxt + 1.f) : 0.f;
            const float a = live ? (float)nxt - (float)t0 : 0.f;
            float span = warp_sum_f(dens);
            span = span > 0.f ? (float)HS_TARGET / span : (float)HS_SPAN;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                span = fminf(fmaxf(span, 2.f), (float)HS_SPAN);
                const float f = warp_sum_f(live ? fminf(fmaxf((span - a) * dens, 0.f), left) : 0.f);
                span *= f > 0.f ? fminf(fmaxf((float)HS_TARGET / f, 0.0625f), 64.f) : 64.f;
            }
            int64_t ispan = (int64_t)fminf(fmaxf(span, 2.f), (float)HS_SPAN);
            int32_t L = 0, nst = 0, t1e = t0;
            for (int guard = 0; guard < 32; ++guard) {
                t1e = (int32_t)min((int64_t)t0 + ispan, (int64_t)it.jhi);
                L = 0;
                if (nxt < t1e) {
                    const float want = ((float)t1e - (float)nxt) * dens * 1.25f + 2.f;
                    L = want >= left ? end - cur : (int32_t)ceilf(want);
                }
                nst = (L + 31) >> 5;
                const int32_t tl = (int32_t)__reduce_add_sync(FULL, (unsigned)L);
                const int32_t ts = (int32_t)__reduce_add_sync(FULL, (unsigned)nst);
                // at span 1 a window holds at most 4 entries: always within bounds
                if ((tl <= HS_CAP && ts <= HS_STEPS) || ispan <= 1) break;
                ispan >>= 1;
            }
            // step table: lane x of the warp then holds load step x
            int32_t sb = nst;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t y = __shfl_up_sync(FULL, sb, d);
                if (lane >= d) sb += y;
            }
            const int32_t nsteps = __shfl_sync(FULL, sb, 31);
            sb -= nst;
            for (int32_t x = 0; x < nst; ++x) {
                const int32_t cnt = min(32, L - 32 * x);
                // the last load of a window that stops short of its range's end
                // bounds the round
                const int32_t bound = (x == nst - 1 && cur + L < end) ? (1 << 16) : 0;
                st_p0[sb + x] = cur + 32 * x;
                st_meta[sb + x] = cnt | (lane << 8) | bound;
            }
            __syncwarp();
            const int32_t my_p0 = lane < nsteps ? st_p0[lane] : 0;
            const int32_t my_meta = lane < nsteps ? st_meta[lane] : 0;
            // 2. loads, HS_GROUP in flight, into the staging buffer
            int32_t cand = (L == 0) ? nxt : INT32_MAX;  // a range without a window
            for (int32_t g0 = 0; g0 < nsteps; g0 += HS_GROUP) {
                int32_t v[HS_GROUP];
#pragma unroll
                for (int b = 0; b < HS_GROUP; ++b) {
                    const int32_t p0 = __shfl_sync(FULL, my_p0, (g0 + b) & 31);
                    const int32_t meta = __shfl_sync(FULL, my_meta, (g0 + b) & 31);
                    const int32_t cnt = (g0 + b < nsteps) ? (meta & 0xff) : 0;
                    v[b] = lane < cnt ? __ldg(&idxTs[p0 + lane]) : INT32_MAX;
                }
#pragma unroll
                for (int b = 0; b < HS_GROUP; ++b) {
                    if (g0 + b >= nsteps) break;
                    const int32_t meta = __shfl_sync(FULL, my_meta, (g0 + b) & 31);
                    stage[(g0 + b) * 32 + lane] = v[b];
                    if ((meta >> 16) && lane == (meta & 0xff) - 1) cand = min(cand, v[b]);
                }
            }
            int32_t t1 = __reduce_min_sync(FULL, cand);
            t1 = (int32_t)min((int64_t)t1, min((int64_t)it.jhi, (int64_t)t0 + HS_SPAN));
            __syncwarp();
            // 3. count the staged entries below t1
            int32_t adv = 0;
            for (int32_t st = 0; st < nsteps; ++st) {
                const int32_t v = stage[st * 32 + lane];
                const int32_t meta = __shfl_sync(FULL, my_meta, st & 31);
                const bool valid = v < t1;
                if (valid) {
                    const uint32_t key = (uint32_t)(v - t0) + 1u;
                    uint32_t h = (key * 2654435761u) >> (32 - HS_LOG);
                    const uint32_t want = (key << 8) | 1u;
                    int probe = 0;
                    for (; probe < HS_SLOTS; ++probe) {
                        const uint32_t old = atomicCAS(&tab[h], 0u, want);
                        if (old == 0u) break;
                        if ((old >> 8) == key) {
                            atomicAdd(&tab[h], 1u);
                            break;
                        }
                        h = (h + 1) & (HS_SLOTS - 1);
                    }
                    if (probe == HS_SLOTS) atomicOr(err, ERR_TABLE);
                }
                const int n = __popc(__ballot_sync(FULL, valid));
                if (lane == ((meta >> 8) & 31)) adv += n;
            }
            if (L > 0) {
                // the first entry not taken is the range's next partner: it sits in
                // the staging buffer at window offset adv (a window that reaches
                // its range's end is taken whole)
                cur += adv;
                nxt = cur >= end ? INT32_MAX : stage[sb * 32 + adv];
            }
            __syncwarp();
            // 4. survivors; the table is cleared as it is read
            int32_t ns = 0;  // fill: survivors staged so far (same in every lane)
#pragma unroll
            for (int r = 0; r < HS_SLOTS / 128; ++r) {
                uint4* t4 = reinterpret_cast<uint4*>(tab) + r * 32 + lane;
                const uint4 w4 = *t4;
                const uint32_t w[4] = {w4.x, w4.y, w4.z, w4.w};
                if (w4.x | w4.y | w4.z | w4.w) *t4 = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const bool sv = w[c] != 0u && (int32_t)(w[c] & 0xffu) >= s;
                    if (!FILL) {
                        my_count += sv ? 1 : 0;
                    } else {
                        const unsigned bal = __ballot_sync(FULL, sv);
                        if (sv) stage[ns + __popc(bal & lt)] = (int32_t)(w[c] - 0x100u);
                        ns += __popc(bal);
                    }
                }
            }
            if (FILL && ns > 0) {
                __syncwarp();
                uint32_t* sv = reinterpret_cast<uint32_t*>(stage);
                warp_sort_u32(sv, ns, lane);
                for (int32_t x = lane; x < ns; x += 32) {
                    const uint32_t w = sv[x];
                    const int64_t p2 = wpos + x;
                    if (p2 < limit) {
                        I[p2] = i - ib;
                        J[p2] = t0 + (int32_t)(w >> 8) - ib;
                        O[p2] = (int32_t)(w & 0xffu);
                    } else {
                        atomicOr(err, ERR_BOUNDS);
                    }
                }
                wpos += ns;
            }
            __syncwarp();
        }
        if (!FILL) {
            const int32_t total = (int32_t)__reduce_add_sync(FULL, (unsigned)my_count);
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
    SLG_CUDA_TRY(cudaFuncSetAttribute(k_sparse_items<false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sp_smem(false)));
}

void wsparse_setup(int sms, int ctas[2]) {
    for (int f = 0; f < 2; ++f) {
        auto kern = f ? k_wsparse_items<true> : k_wsparse_items<false>;
        SLG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)HS_SMEM));
        int d = 0;
        SLG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, kern, HS_WARPS * 32, HS_SMEM));
        ctas[f] = sms * (d > 0 ? d : 1);
    }
}

void launch_wsparse(bool fill, int ctas, const GraphDev& g, const Plan& p, RowS rs,
                    int32_t item_lo, int32_t item_hi, int32_t* icnt, const int64_t* ioff,
                    int32_t* I, int32_t* J, int32_t* O, int32_t* queue, int64_t limit,
                    int32_t* err, cudaStream_t st) {
    if (fill)
        k_wsparse_items<true><<<ctas, HS_WARPS * 32, HS_SMEM, st>>>(
            p.items, p.mode_list[MODE_WSPARSE], p.mode_rank[MODE_WSPARSE], item_lo, item_hi,
            g.off, p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I, J, O, queue, limit, err);
    else
        k_wsparse_items<false><<<ctas, HS_WARPS * 32, HS_SMEM, st>>>(
            p.items, p.mode_list[MODE_WSPARSE], p.mode_rank[MODE_WSPARSE], item_lo, item_hi,
            g.off, p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I, J, O, queue, limit, err);
    SLG_LAUNCH_CHECK();
}

void launch_sparse(bool fill, int ctas, const GraphDev& g, const Plan& p, RowS rs,
                   int32_t item_lo, int32_t item_hi, int32_t* icnt, const int64_t* ioff,
                   int32_t* I, int32_t* J, int32_t* O, int32_t* queue, int64_t limit,
                   int32_t* err, cudaStream_t st, const StageArgs& sa, const EnsArgs* ens4) {
    if (fill)
        k_sparse_items<true><<<ctas, SP_THREADS, sp_smem(true), st>>>(
            p.items, p.mode_list[MODE_SPARSE], p.mode_rank[MODE_SPARSE], item_lo, item_hi, g.off,
            p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I, J, O, queue, limit, err, sa, nullptr);
    else if (ens4)
        k_sparse_items<false, true><<<ctas, SP_THREADS, sp_smem(false), st>>>(
            p.items, p.mode_list[MODE_SPARSE], p.mode_rank[MODE_SPARSE], item_lo, item_hi, g.off,
            p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I, J, O, queue, limit, err, StageArgs{}, ens4);
    else
        k_sparse_items<false><<<ctas, SP_THREADS, sp_smem(false), st>>>(
            p.items, p.mode_list[MODE_SPARSE], p.mode_rank[MODE_SPARSE], item_lo, item_hi, g.off,
            p.wbeg, p.wend, p.idxTs, rs, icnt, ioff, I, J, O, queue, limit, err, StageArgs{},
            nullptr);
    SLG_LAUNCH_CHECK();
}

}  // namespace slg
