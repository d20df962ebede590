// Internal declarations of libslg (not part of the C ABI).
//
// Terms used throughout (Liu et al., arXiv 2201.11326):
//   row i        hyperedge e_i; its CSR row lists its vertices (Section II-A)
//   adj(v)       hyperedges containing vertex v, ascending (the dual, H^T)
//   E_s          hyperedges with |e| >= s (Section II-B)
//   wedge        (i, v, j) with i < j, v in e_i ∩ e_j, |e_i|, |e_j| >= s: one
//                increment of Algorithm 2's overlap counter (Section III-C)
//   adj_s(v)     adj(v) restricted to E_s ("pruned transpose")
//   wedge range  for incidence (i, v): the suffix of adj_s(v) after i, i.e.
//                the j of every wedge (i, v, j)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "slg.h"

namespace slg {

// ---------------------------------------------------------------- status

struct Error {
    slg_status code;
    std::string msg;
};

void set_error(slg_status code, const std::string& msg);

#define SLG_CUDA_TRY(expr)                                                         \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            throw ::slg::Error{e_ == cudaErrorMemoryAllocation ? SLG_ENOMEM        \
                                                                : SLG_ECUDA,       \
                               std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
        }                                                                          \
    } while (0)

// Every kernel launch of the library is followed by SLG_LAUNCH_CHECK(), which
// also counts it (reported by slg_kernel_launches()).
void count_launch();
// Bytes of staging pools held by all handles (plan_staging, Plan::release_stage).
void stage_bytes_add(int64_t d);
#define SLG_LAUNCH_CHECK()                    \
    do {                                      \
        ::slg::count_launch();                \
        SLG_CUDA_TRY(cudaGetLastError());     \
    } while (0)

// Stream-ordered device allocation (released in stream order; a null pointer
// is ignored, and a failed release is not reported: it runs on cleanup paths).
template <typename T>
T* dalloc(size_t count, cudaStream_t st) {
    T* p = nullptr;
    SLG_CUDA_TRY(cudaMallocAsync((void**)&p, sizeof(T) * (count ? count : 1), st));
    return p;
}

template <typename T>
void dfree(T*& p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
}

// ------------------------------------------------------------ work items
//
// A work item is one row i restricted to candidate partners j in [jlo, jhi).
// Items of a row are contiguous, in increasing j, and cover every wedge of
// the row; items of different rows follow row order. The canonical output is
// therefore the concatenation of the items' outputs in item order.

enum ItemMode : int32_t {
    MODE_WARP = 0,   // whole row, few wedges: one warp, small hash table
    MODE_BLOCK = 1,  // sparse slice: one CTA, shared-memory hash table
    MODE_DENSE = 2,  // dense slice, many non-hub ranges: one CTA, j tiles of 32768
    MODE_WDENSE = 3, // dense slice, <= 32 non-hub ranges: one warp, j tiles of 4096
    MODE_SPARSE = 4, // sparse slice of a heavy row (|e_i| <= 255): one CTA, j tiles of
                     // 65536 8-bit counters and a list of the counters it touched
    MODE_WSPARSE = 5,// the same for rows with |e_i| <= 32: one warp, counting in hash rounds
    MODE_HUBPAIR = 6,// sparse row at s >= 2 whose candidates come from its non-hub wedges and
                     // the rows sharing a pair of its hubs: one CTA, shared-memory hash table
    NMODES = 7
};

struct Item {
    int32_t row;
    int32_t jlo;
    int32_t jhi;
    int32_t mode;
};

// Threshold and output-id base of a row. A single graph has one s for all
// rows and its ids start at 0; a batch (disjoint union of graphs, each with
// its own s) has per-row values, and ids are written relative to the first
// row of the row's own graph.
struct RowS {
    const int32_t* srow;   // per-row s, or null: every row uses s
    const int32_t* rbase;  // first row of the row's graph, or null: 0
    int32_t s;
    __device__ __forceinline__ int32_t s_of(int32_t i) const { return srow ? srow[i] : s; }
    __device__ __forceinline__ int32_t base_of(int32_t i) const { return rbase ? rbase[i] : 0; }
};

// Per-handler kernel timing (CUDA events on the graph's stream), for the
// counting pass [0] and the fill pass [1].
struct ModeTimer {
    bool on = false;
    cudaEvent_t ev[2 * NMODES] = {};
    float ms[2][NMODES] = {};
    int64_t launches[2][NMODES] = {};
    cudaEvent_t fev[2] = {};  // around one ensemble list filter
};

// Tunables of the binning (chosen per graph; defaults in plan.cu).
struct BinParams {
    int32_t warp_max_wedges;   // rows with W_i <= this go to MODE_WARP
    int32_t block_item_wedges; // target wedges per MODE_BLOCK item
    int32_t dense_min_density; // dense when 256*W_i >= density*span (density/256)
    int32_t dense_item_tiles;  // tiles per MODE_DENSE item (x4096 ids per MODE_WDENSE item)
    int32_t wdense_max_ranges; // rows with at most this many non-hub wedge ranges (<= 32)
                               // use the warp-level dense handler; 0 disables it
    int32_t sparse_min_per_tile;  // a non-dense row with |e_i| <= 255 and at least this many
                                  // wedges per 65536-id tile of its span goes to MODE_SPARSE
                                  // (< 0 disables it)
    int32_t sparse_item_wedges;   // target wedges per MODE_SPARSE / MODE_WSPARSE item
    int32_t wsparse_max_size;     // sparse rows with |e_i| <= this (<= 32) use the warp-level
                                  // accumulator; 0 disables it
};

// ---------------------------------------------------------- kernel sizes

constexpr int WARP_TABLE = 256;           // slots per warp table (MODE_WARP)
constexpr int WARP_CTA_WARPS = 8;         // warps per CTA in MODE_WARP
constexpr int BLOCK_THREADS = 512;        // MODE_BLOCK CTA
constexpr int BLOCK_TABLE = 4096;         // slots per CTA table (MODE_BLOCK)
constexpr int BLOCK_CAP = BLOCK_TABLE / 2;// distinct keys before a slice splits
constexpr int DENSE_THREADS = 512;        // MODE_DENSE CTA
constexpr int DENSE_TILE = 32768;         // j per tile (16-bit counters)
constexpr int DENSE_MAXE = 1024;          // incidences a dense row may have
constexpr int MAX_HUBS = 32;              // vertices summarised by per-row bit masks
constexpr int WD_WARPS = 12;              // warps per CTA in MODE_WDENSE
constexpr int WD_TILE = 4096;             // j per warp tile (8-bit counters, 4 KB)
constexpr int WD_ITEM = 8192;             // j per MODE_WDENSE item = WD_ITEM * dense_item_tiles
constexpr int WD_MAXR = 32;               // non-hub wedge ranges a MODE_WDENSE row may have
constexpr int DENSE_MAX_SIZE = 65535;     // |e_i| bound for 16-bit counters
constexpr int ENS_MAX = 16;               // thresholds in one ensemble (Algorithm 3)
constexpr int SP_THREADS = 512;           // MODE_SPARSE CTA
constexpr int SP_TILE = 65536;            // j per tile (8-bit counters, 64 KB)
constexpr int SP_TOUCH = 8192;            // touched counters listed per tile
constexpr int SP_MAX_SIZE = 255;          // |e_i| bound for 8-bit counters
constexpr int WS_MAXE = 32;               // |e_i| bound of MODE_WSPARSE (one range per lane)
constexpr int HP_MAXK = 4096;             // hubs of the hub-pair index (MODE_HUBPAIR)
constexpr int HP_ITEM = 2304;             // entries (non-hub wedges + pair-list hits) per item
constexpr int HP_MAXR = 256;              // hub-pair incidences of a MODE_HUBPAIR row, at most

// --------------------------------------------------------- device helpers

__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
    // SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ inline uint64_t pair_digest(int32_t i, int64_t k, int32_t j, int32_t o) {
    uint64_t a = splitmix64(((uint64_t)(uint32_t)i << 32) | (uint64_t)(uint32_t)k);
    return splitmix64(a ^ (((uint64_t)(uint32_t)j << 32) | (uint64_t)(uint32_t)o));
}

// ------------------------------------------------------ host-side launches
//
// Each returns after enqueueing on `st`; scratch comes from stream-ordered
// allocation (cudaMallocAsync) and is released in stream order.

// exclusive scan: out[0..n] with out[n] = total (out has n+1 entries)
void scan_i32_to_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st);
void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t st);
void scan_i64_to_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st);

// load-time kernels (transpose.cu)
void launch_validate(const int32_t* off, const int32_t* idx, int32_t m, int32_t n, int64_t nnz,
                     int32_t* rowid, int32_t* size, int32_t* flag, cudaStream_t st);
void build_transpose(const int32_t* idx, const int32_t* rowid, int32_t n, int64_t nnz,
                     int32_t* offT, int32_t* idxT, int32_t* tpos, cudaStream_t st);
// Hub vertices (at most MAX_HUBS, highest degree first) and per-row masks.
// Returns the number of hubs.
int32_t build_hubs(const int32_t* off, const int32_t* idx, const int32_t* offT, int32_t m,
                   int32_t n, int32_t* hubidx, uint32_t* hubmask, cudaStream_t st);

}  // namespace slg
