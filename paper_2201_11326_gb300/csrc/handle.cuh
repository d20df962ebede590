// The graph handle behind the C ABI's opaque slg_graph (internal).
#pragma once

#include <vector>

#include "plan.cuh"

namespace slg {

BinParams default_bins();

// CUDA events around the phases of the last counting pass / fill.
struct Timer {
    bool on = false;
    cudaEvent_t ev[6] = {};
    void init();
    void mark(int k, cudaStream_t st);
    void destroy();
};

void mtimer_init(ModeTimer& t);

}  // namespace slg

struct slg_graph {
    slg::GraphDev g;
    bool owns_data = true;  // false for a view sharing another handle's arrays
    slg::Plan plan;
    cudaStream_t st = nullptr;
    int device = 0;
    slg::BinParams bp = slg::default_bins();
    slg::Timer timer;
    slg::ModeTimer mtimer;
    float ms[5] = {0, 0, 0, 0, 0};
    std::vector<int32_t> batch_row_base;  // members' first rows (k+1) when this is a batch
    // hub pairs (MODE_HUBPAIR): built on the first plan for s >= 2 whose table
    // and sparse-accumulator rows carry at least hp_min_wedges wedges
    slg::HubPairs hp;
    int32_t hp_max_hubs = slg::HP_MAXK;           // 0 disables the hub-pair handler
    int64_t hp_min_wedges = (int64_t)1 << 33;
    int64_t hp_max_pairs = (int64_t)1900000000;  // hub-pair incidences at most
    // staging pool of the counting pass (slg::StageArgs): -1 automatic, 0 off,
    // > 0 at most this many bytes
    int64_t stage_max_bytes = -1;
    // an ensemble's window of every list: list t from list t-1 by filtering (1),
    // by walking its rows (0), or whichever reads less (-1)
    int32_t ens_filter = -1;
    // per ensemble list index, over windows of every list: {windows walked,
    // pairs walked, windows filtered, pairs filtered, filter device time in
    // microseconds while timing is on, pairs the filter read}
    // (slg_ensemble_fill_stats)
    int64_t ens_made[slg::ENS_MAX][6] = {};
};

namespace slg {

// A handle that shares base's device arrays (which must outlive it) with its
// own plan and stream, so that several s of one graph can run concurrently.
slg_graph* make_view(const slg_graph* base, cudaStream_t st);

// Builds h->plan for s (s = 0: a batch's own thresholds), deciding on the way
// whether the hub-pair handler applies and building the hub pairs when it does.
void build_plan(slg_graph* h, int32_t s, const BinParams& bp);

// Chooses h->bp for s by timing binnings on h (autotune.cu); the plan is left
// released.
void autotune(slg_graph* h, int32_t s, int32_t max_trials, float* best_ms);

// Whether h's plan has rows a staging pool serves (and h may stage).
bool can_stage(const slg_graph* h);
// A staging pool for h's plan of at most `want` pairs in chunks of `chunk`,
// within the device-memory budget; false (no pool) when too little fits.
bool alloc_stage(slg_graph* h, int64_t want, int64_t chunk);

// The next window of one-walk construction (stream.cu): rows r0 .. *r1 of the
// lists for s[0..k-1], back to back in I/J/O (device, cap pairs), pairs[t]
// each. Builds the plan and its bounds on first use.
void stream_window(slg_graph* h, const int32_t* s, int32_t k, int32_t r0, int32_t* I,
                   int32_t* J, int32_t* O, int64_t cap, int32_t* r1, int64_t* pairs);

}  // namespace slg
