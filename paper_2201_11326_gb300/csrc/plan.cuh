// Device-resident graph and per-s plan (internal).
#pragma once

#include "slg_internal.cuh"

namespace slg {

// A loaded hypergraph: the caller's CSR, its dual, and per-incidence tables.
struct GraphDev {
    int32_t m = 0, n = 0;
    int64_t nnz = 0;
    int32_t min_size = 0;   // smallest |e_i| over non-empty rows (0 if none)
    int32_t max_size = 0;   // largest |e_i|
    int32_t* off = nullptr;    // [m+1]
    int32_t* idx = nullptr;    // [nnz]
    int32_t* size = nullptr;   // [m]   |e_i|
    int32_t* rowid = nullptr;  // [nnz] row of incidence e
    int32_t* offT = nullptr;   // [n+1] H^T offsets
    int32_t* idxT = nullptr;   // [nnz] adj(v) ascending
    int32_t* tpos = nullptr;   // [nnz] position of incidence e inside H^T
    int32_t* srow = nullptr;   // [m] per-row s of a batch (null for a single graph)
    int32_t* rbase = nullptr;  // [m] first row of the row's graph in a batch
    int32_t nhubs = 0;
    int32_t* hubidx = nullptr;     // [n]  hub number of vertex v, -1 if none
    uint32_t* hubmask = nullptr;   // [m]  bit b set when hub b is in e_i
};

// Hub pairs of a graph (built on demand for s >= 2, when its sparse rows carry
// many wedges). The HP hubs are the (at most max_hubs) highest-degree vertices,
// numbered in vertex order. For a row i with hubs H_i, its hub-pair incidences
// are the keys a*K + b of the pairs a < b of H_i (ascending), and the
// transpose lists, for each pair key, the rows holding both hubs in increasing
// id. Two rows then share t >= 2 hubs exactly when each lies in t(t-1)/2 of
// the other's pair lists.
struct HubPairs {
    bool built = false, tried = false;
    int32_t K = 0;             // hubs
    int64_t E1 = 0, E2 = 0;    // hub incidences, hub-pair incidences
    int32_t* hp_id = nullptr;  // [n] hub number of v (vertex order), -1 if none
    int32_t* hoff = nullptr;   // [m+1] row hub lists
    int32_t* hlist = nullptr;  // [E1] hub numbers of each row, ascending
    int32_t* off2 = nullptr;   // [m+1] row hub-pair incidences
    int32_t* idx2 = nullptr;   // [E2] pair keys, ascending per row
    int32_t* offT2 = nullptr;  // [K*K+1] pair lists
    int32_t* idxT2 = nullptr;  // [E2] rows of each pair list, ascending
    int32_t* tpos2 = nullptr;  // [E2] position of each hub-pair incidence in idxT2
    // rows with more than bigk hubs also keep their hubs as a bitmap of K bits
    int32_t bigk = 0;
    int32_t* bigidx = nullptr;    // [m] bitmap number of the row, -1 if none
    uint32_t* bigbits = nullptr;  // [rows with a bitmap][HP_MAXK / 32]
    // per row, 64 bytes read in one go by a one-hub look: 32 16-bit fields,
    // the row's hub count then its hub numbers (count 0xffff: more than 31)
    uint4* hrec = nullptr;        // [m][4]
    void release(cudaStream_t st);
};

// Builds hp for g with at most max_hubs hubs and at most max_pairs hub-pair
// incidences (fewer hubs when needed); leaves hp unbuilt (tried) when no hub
// pair exists.
void hubpair_build(const GraphDev& g, int32_t max_hubs, int64_t max_pairs, HubPairs& hp,
                   cudaStream_t st);

// Device descriptor of one member of a batch.
struct BatchPart {
    const int32_t* off;
    const int32_t* idx;
    const int32_t* size;
    const int32_t* rowid;
    const int32_t* offT;
    const int32_t* idxT;
    const int32_t* tpos;
    const int32_t* hubidx;
    const uint32_t* hubmask;
    int32_t m, n;
    int64_t nnz;
    int32_t row_base, vert_base;
    int64_t nnz_base;
    int32_t s;
};

// Writes the disjoint union of the members into `out` (arrays preallocated:
// off[M+1], idx/rowid/idxT/tpos[NNZ], size/srow/rbase/hubmask[M], offT[N+1],
// hubidx[N]).
void launch_concat(const BatchPart* parts_dev, int32_t k, int32_t M, int32_t N, int64_t NNZ,
                   const GraphDev& out, cudaStream_t st);
// Per member b of a batch: wsum[b] = sum of W over its rows, dsum[b] = sum of
// rowdig over its rows (mod 2^64; rowdig may be null, dsum is then 0).
void launch_member_sums(const int64_t* W, const unsigned long long* rowdig,
                        const int32_t* row_base_dev, int32_t k, long long* wsum_dev,
                        unsigned long long* dsum_dev, cudaStream_t st);
// out[b] = rowoff[row_base[b]] for b = 0..k
void launch_gather_offsets(const int64_t* rowoff, const int32_t* row_base_dev, int32_t k,
                           int64_t* out_dev, cudaStream_t st);

// Everything derived for one s. Items and offsets are valid once built;
// icnt/ioff/rowoff once `counted`.
// The thresholds of an ensemble counted in one pass (Algorithm 3): list t
// holds the pairs with overlap >= s[t]; k = 0 for a single threshold.
struct EnsArgs {
    int32_t k = 0;                   // number of lists (0: one threshold, from RowS)
    int32_t s[ENS_MAX] = {};         // thresholds, strictly ascending
    uint32_t bias[ENS_MAX] = {};     // 0x01010101 * (128 - min(s[t], 128)) (byte-wise compares)
    int32_t* icnt = nullptr;         // per-item counts of list t at [t * stride]
    int64_t stride = 0;
};

// A staging pool for the counting pass: the sparse-accumulator and hub-pair
// fill kernels, run as the counting pass, write each item's pairs (in order)
// into per-CTA chunks of the pool as well as its count; an item whose pairs
// all fit is staged at at[q], and a window later copies it into place instead
// of walking it again. J == nullptr: no staging writes (a window's fill, which
// skips the items with at[q] >= 0 when at is given).
constexpr int64_t SG_CHUNK = 1 << 20;  // pairs a CTA takes from the pool at a time, at most
struct StageArgs {
    int32_t* J = nullptr;                  // staged partners (member-local ids)
    uint8_t* O = nullptr;                  // staged overlaps (<= 255: both handlers take
                                           // rows of at most 255 vertices)
    int64_t cap = 0;                       // pool size in pairs
    unsigned long long* cursor = nullptr;  // next free pair of the pool
    int64_t* at = nullptr;                 // [nitems] first staged pair of item q, -1: not staged
    int64_t chunk = SG_CHUNK;              // pairs a CTA takes from the pool at a time
    int64_t min_room = SG_CHUNK / 32;      // an item starts in a fresh chunk below this room
};

struct Plan {
    int32_t s = 0;              // 0 for a batch (per-row s)
    bool built = false;
    RowS rs{};                  // thresholds and id bases used by the kernels
    int32_t* ks = nullptr;      // [nnz+1] kept-prefix over H^T positions (null when nothing is pruned)
    int32_t* idxTs = nullptr;   // pruned H^T (aliases idxT when nothing is pruned)
    bool idxTs_owned = false;
    int32_t* wbeg = nullptr;    // [nnz] wedge range of incidence e in idxTs
    int32_t* wend = nullptr;
    int64_t* W = nullptr;       // [m] wedges of row i
    int32_t* jmin = nullptr;    // [m] first / last candidate partner of row i
    int32_t* jmax = nullptr;
    int32_t* nnh = nullptr;     // [m] non-hub incidences of row i with a non-empty wedge range
    int32_t* row_item = nullptr;  // [m+1] first item of row i
    int64_t nitems = 0;
    Item* items = nullptr;
    int32_t* mode_rank[NMODES] = {};  // [nitems+1]
    int32_t* mode_list[NMODES] = {};  // item ids per mode, ascending
    int64_t mode_count[NMODES] = {};
    int32_t* icnt = nullptr;    // [nitems] pairs per item
    int64_t* ioff = nullptr;    // [nitems+1] output offset per item
    int64_t* rowoff = nullptr;  // [m+1] output offset per row
    bool counted = false;
    int64_t pairs = 0;
    int64_t wedges = 0;

    // Ensemble (Algorithm 3, Section III-D): thresholds s[0] < ... < s[k-1]
    // counted over this plan, which is built for s[0]. List t of a row holds
    // its partners with overlap >= s[t]; per list, counts and offsets as above.
    struct Ensemble {
        int32_t k = 0;
        int32_t s[ENS_MAX] = {};
        int32_t* icnt = nullptr;    // [k][nitems]
        int64_t* ioff = nullptr;    // [k][nitems+1]
        int64_t* rowoff = nullptr;  // [k][m+1]
        int64_t* rowtot = nullptr;  // [m+1] sum of the k row offsets (window planning)
        int64_t pairs[ENS_MAX] = {};
        bool counted = false;
    } ens;

    // hub pairs for s (MODE_HUBPAIR rows; null when the plan uses none)
    const HubPairs* hp = nullptr;
    int32_t* ks2 = nullptr;      // [E2+1] kept-prefix over the pair lists (null: nothing pruned)
    int32_t* idxT2s = nullptr;   // pruned pair lists (aliases hp->idxT2 when nothing is pruned)
    bool idxT2s_owned = false;
    int32_t* wbeg2 = nullptr;    // [E2] wedge range of each hub-pair incidence in idxT2s
    int32_t* wend2 = nullptr;
    int64_t* Wp = nullptr;       // [m] entries a MODE_HUBPAIR row walks (non-hub wedges +
                                 // pair-list hits); null without hub pairs

    // staged counting (see StageArgs); null when the counting pass stages nothing
    int64_t* stage_at = nullptr;   // [nitems]
    int32_t* stage_J = nullptr;    // [stage_cap]
    uint8_t* stage_O = nullptr;    // [stage_cap]
    unsigned long long* stage_cursor = nullptr;
    int64_t stage_cap = 0;
    int64_t stage_chunk = SG_CHUNK;
    int32_t stage_s = -1;  // the threshold whose list the last counting pass staged
    int64_t stage_bytes = 0;  // device bytes of the pool and its item positions
    StageArgs stage_args() const {
        return StageArgs{stage_J, stage_O, stage_cap, stage_cursor, stage_at, stage_chunk,
                         stage_chunk / 32};
    }
    void release_stage(cudaStream_t st);

    // one-walk windows (stream_window): their thresholds, the cumulative bound
    // on each row's list-0 pairs, and what the last window observed
    int64_t* stream_cum = nullptr;  // [m+1]
    int32_t stream_k = 0;
    int32_t stream_s[ENS_MAX] = {};
    double stream_lambda = 1.0;  // list-0 pairs per unit of bound
    double stream_phi = 1.0;     // pairs of every list per list-0 pair
    void release_stream(cudaStream_t st);

    RowS rs_for(int32_t s_t) const { return RowS{rs.srow, rs.rbase, s_t}; }
    void release_ensemble(cudaStream_t st);
    void release(cudaStream_t st);
};

// hp: hub pairs to bin sparse rows into MODE_HUBPAIR (s >= 2), or null.
void plan_build(const GraphDev& g, int32_t s, const BinParams& bp, Plan& p, cudaStream_t st,
                const HubPairs* hp = nullptr);
// Wedges of the rows binned as table or sparse-accumulator rows (MODE_BLOCK,
// MODE_SPARSE, MODE_WSPARSE) in a built plan: what hub pairs could shorten.
int64_t plan_sparse_wedges(const GraphDev& g, const Plan& p, cudaStream_t st);
void plan_offsets(const GraphDev& g, Plan& p, cudaStream_t st);
// Pairs the sparse-accumulator and hub-pair rows can have at most (the
// entries they walk): what a staging pool may need to hold.
int64_t plan_stage_bound(const GraphDev& g, const Plan& p, cudaStream_t st);
// Items the last counting pass staged.
int64_t plan_staged_items(const Plan& p, cudaStream_t st);
// Largest row total and window splits over cumulative row offsets rowoff[m+1]
// (a single list's or the ensemble's sum).
int64_t plan_max_row(const GraphDev& g, const int64_t* rowoff, cudaStream_t st);
int32_t plan_windows(const GraphDev& g, const int64_t* rowoff, int64_t C, int32_t* splits_dev,
                     cudaStream_t st);
// Counts and offsets of every list of an ensemble (the plan is built for s[0]).
void ensemble_count(const GraphDev& g, Plan& p, const int32_t* s, int32_t k, ModeTimer* mt,
                    cudaStream_t st);

// Counting and filling (count_fill.cu). Items [item_lo, item_hi) are filled
// into I/J/O at position ioff[q] - ioff[item_lo].
// `rs` carries the threshold (the plan's own, or one of an ensemble's), icnt
// and ioff the matching per-item counts and offsets.
void run_count(const GraphDev& g, const Plan& p, RowS rs, int32_t* icnt, ModeTimer* mt,
               cudaStream_t st);
// Staged items of a list: the pool's per-item counts come from st_ioff (the
// list's item offsets; null: nothing of this list is staged).
struct StageUse {
    const int64_t* st_ioff = nullptr;
};
// Staged items (see StageUse) are copied into place and the fill kernels skip
// them.
void run_fill(const GraphDev& g, const Plan& p, RowS rs, const int64_t* ioff, int32_t item_lo,
              int32_t item_hi, int32_t* I, int32_t* J, int32_t* O, int64_t limit, ModeTimer* mt,
              cudaStream_t st, StageUse su = StageUse{});
// Counting pass of the handlers in the bit set `modes` only, over every item.
void run_count_modes(const GraphDev& g, const Plan& p, RowS rs, unsigned modes, int32_t* icnt,
                     ModeTimer* mt, cudaStream_t st);
// Counting pass of the sparse-accumulator and hub-pair items of
// [item_lo, item_hi): their fill kernels count and stage while the plan's pool
// lasts (stage_at of the range reset first), the counting kernels take the rest.
void run_count_staged(const GraphDev& g, const Plan& p, RowS rs, int32_t item_lo, int32_t item_hi,
                      int32_t* icnt, ModeTimer* mt, cudaStream_t st);
// The pairs of one list with overlap >= s, in order, into I2/J2/O2 when they
// are at most `room` (and I2 is not null); returns their number either way.
int64_t run_filter_room(const int32_t* I, const int32_t* J, const int32_t* O, int64_t n, int32_t s,
                        int32_t* I2, int32_t* J2, int32_t* O2, int64_t room, cudaStream_t st);
// The pairs of one list with overlap >= s (n in, expect out, order kept): a list
// of an ensemble from the list before it.
void run_filter(const int32_t* I, const int32_t* J, const int32_t* O, int64_t n, int32_t s,
                int32_t* I2, int32_t* J2, int32_t* O2, int64_t expect, cudaStream_t st);
// Entries a walk of rows [r0, r1) of the plan reads: wedges through vertices
// that are not mask hubs, and the walked entries of hub-pair rows.
int64_t plan_row_walk(const GraphDev& g, const Plan& p, int32_t r0, int32_t r1, cudaStream_t st);
// Ensemble counting pass over the plan's items (p.ens.k lists, thresholds
// p.ens.s): counts into p.ens.icnt. Lists are filled one at a time by run_fill.
void run_count_ensemble(const GraphDev& g, const Plan& p, ModeTimer* mt, cudaStream_t st);
// Sparse-accumulator handler (sparse.cu): kernel attributes and CTAs per
// launch (count, fill), and one launch over the MODE_SPARSE items.
void sparse_setup(int sms, int ctas[2]);
void wsparse_setup(int sms, int ctas[2]);
void launch_wsparse(bool fill, int ctas, const GraphDev& g, const Plan& p, RowS rs,
                    int32_t item_lo, int32_t item_hi, int32_t* icnt, const int64_t* ioff,
                    int32_t* I, int32_t* J, int32_t* O, int32_t* queue, int64_t limit,
                    int32_t* err, cudaStream_t st);
void launch_sparse(bool fill, int ctas, const GraphDev& g, const Plan& p, RowS rs,
                   int32_t item_lo, int32_t item_hi, int32_t* icnt, const int64_t* ioff,
                   int32_t* I, int32_t* J, int32_t* O, int32_t* queue, int64_t limit,
                   int32_t* err, cudaStream_t st, const StageArgs& sa = StageArgs{},
                   const EnsArgs* ens4 = nullptr);
// Per-handler totals over rows (needs counts): rows, wedges, incidences, pairs,
// non-hub wedges, partners scanned by the dense extraction (count, fill).
constexpr int MS_COLS = 7;
// rowoff/ioff: the list's row and item offsets (null: the plan's own).
void plan_mode_stats(const GraphDev& g, const Plan& p, int64_t out[NMODES][MS_COLS],
                     cudaStream_t st, const int64_t* rowoff = nullptr,
                     const int64_t* ioff = nullptr);
// Hub-pair handler (hubpair.cu): kernel attributes, CTAs per launch, and one
// launch over the MODE_HUBPAIR items.
void hubpair_setup(int sms, int ctas[2]);
void launch_hubpair(bool fill, int ctas, const GraphDev& g, const Plan& p, RowS rs,
                    int32_t item_lo, int32_t item_hi, int32_t* icnt, const int64_t* ioff,
                    int32_t* I, int32_t* J, int32_t* O, int32_t* queue, int64_t limit,
                    int32_t* err, cudaStream_t st, const StageArgs& sa = StageArgs{},
                    const EnsArgs* ens4 = nullptr);
// Digest of a filled window (rows [r0, r1), pairs at I/J/O[0..P)).
void run_digest(RowS rs, const int64_t* rowoff, int32_t r0, int32_t r1, const int32_t* I,
                const int32_t* J, const int32_t* O, int64_t P, unsigned long long* total_dev,
                unsigned long long* rows_dev, cudaStream_t st);

}  // namespace slg
