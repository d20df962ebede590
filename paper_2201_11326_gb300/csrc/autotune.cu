// Autotuning of the binning thresholds (the knobs of slg_set_bins).
//
// The paper tunes its own machine by hand: blocked or cyclic ranges, chunk
// sizes and relabel-by-degree (Sections III-F and IV). Here the knobs are the
// work-item shapes and handler thresholds of the binning, and they are chosen
// per graph by measurement: coordinate descent from the defaults, one knob at
// a time over a short list of values. A trial is the planning, the counting pass
// and the fill of a fixed sample of row windows, timed with CUDA events on the
// graph's stream. Results never depend on the thresholds, only the time does.
#include <cstdio>
#include <vector>

#include "handle.cuh"

namespace slg {
namespace {

constexpr int64_t SAMPLE_PAIRS = (int64_t)1 << 26;  // fill sample: 768 MiB of I/J/O
constexpr int SAMPLE_WINDOWS = 8;

struct Knob {
    int32_t BinParams::*field;
    std::vector<int32_t> values;
};

// Row windows spread over the graph whose pairs add up to at most
// SAMPLE_PAIRS: window w starts at row w*m/SAMPLE_WINDOWS and takes rows while
// they fit its share. A row with more pairs than the share is left out.
std::vector<std::pair<int32_t, int32_t>> sample_rows(const std::vector<int64_t>& rowoff,
                                                     int32_t m) {
    std::vector<std::pair<int32_t, int32_t>> out;
    const int64_t share = SAMPLE_PAIRS / SAMPLE_WINDOWS;
    int32_t prev_end = 0;
    for (int w = 0; w < SAMPLE_WINDOWS; ++w) {
        int32_t r0 = (int32_t)((int64_t)m * w / SAMPLE_WINDOWS);
        if (r0 < prev_end) r0 = prev_end;
        int32_t r1 = r0;
        while (r1 < m && rowoff[r1 + 1] - rowoff[r0] <= share) ++r1;
        if (r1 > r0) out.emplace_back(r0, r1);
        prev_end = r1;
    }
    return out;
}

}  // namespace

// Times one binning on h: plan for s, counting pass, offsets, and the fill of
// the sample windows into I/J/O. Returns milliseconds.
float autotune_trial(slg_graph* h, int32_t s, const BinParams& bp,
                     const std::vector<std::pair<int32_t, int32_t>>& sample, int32_t* I,
                     int32_t* J, int32_t* O, cudaEvent_t e0, cudaEvent_t e1) {
    Plan& p = h->plan;
    p.release(h->st);
    SLG_CUDA_TRY(cudaEventRecord(e0, h->st));
    build_plan(h, s, bp);
    run_count(h->g, p, p.rs, p.icnt, nullptr, h->st);
    plan_offsets(h->g, p, h->st);
    for (const auto& w : sample) {
        int32_t q[2];
        int64_t o[2];
        SLG_CUDA_TRY(cudaMemcpyAsync(&q[0], p.row_item + w.first, 4, cudaMemcpyDeviceToHost, h->st));
        SLG_CUDA_TRY(cudaMemcpyAsync(&q[1], p.row_item + w.second, 4, cudaMemcpyDeviceToHost, h->st));
        SLG_CUDA_TRY(cudaMemcpyAsync(&o[0], p.rowoff + w.first, 8, cudaMemcpyDeviceToHost, h->st));
        SLG_CUDA_TRY(cudaMemcpyAsync(&o[1], p.rowoff + w.second, 8, cudaMemcpyDeviceToHost, h->st));
        SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
        run_fill(h->g, p, p.rs, p.ioff, q[0], q[1], I, J, O, o[1] - o[0], nullptr, h->st);
    }
    SLG_CUDA_TRY(cudaEventRecord(e1, h->st));
    SLG_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0;
    SLG_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    return ms;
}

// Coordinate descent over the knobs, at most max_trials trials (the first is
// the current binning). Leaves the best binning in h->bp, the plan released.
void autotune(slg_graph* h, int32_t s, int32_t max_trials, float* best_ms_out) {
    const int32_t m = h->g.m;
    // per-row counts do not depend on the binning: take the sample from the
    // current one
    h->plan.release(h->st);
    build_plan(h, s, h->bp);
    run_count(h->g, h->plan, h->plan.rs, h->plan.icnt, nullptr, h->st);
    plan_offsets(h->g, h->plan, h->st);
    std::vector<int64_t> rowoff((size_t)m + 1);
    SLG_CUDA_TRY(cudaMemcpyAsync(rowoff.data(), h->plan.rowoff, sizeof(int64_t) * ((size_t)m + 1),
                                 cudaMemcpyDeviceToHost, h->st));
    SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
    const auto sample = sample_rows(rowoff, m);
    int32_t* buf = dalloc<int32_t>((size_t)3 * SAMPLE_PAIRS, h->st);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SLG_CUDA_TRY(cudaEventCreate(&e0));
    SLG_CUDA_TRY(cudaEventCreate(&e1));
    int32_t *I = buf, *J = buf + SAMPLE_PAIRS, *O = buf + 2 * SAMPLE_PAIRS;

    const std::vector<Knob> knobs = {
        {&BinParams::dense_item_tiles, {1, 2, 4, 8, 16}},
        {&BinParams::dense_min_density, {16, 32, 64, 128, 256}},
        {&BinParams::sparse_min_per_tile, {-1, 16, 64, 256}},
        {&BinParams::sparse_item_wedges, {16384, 65536, 262144}},
        {&BinParams::wdense_max_ranges, {8, 16, 32}},
        {&BinParams::block_item_wedges, {256, 1024, 4096}},
        {&BinParams::warp_max_wedges, {32, 64, 128}},
        {&BinParams::wsparse_max_size, {0, 16, 32}},
    };
    BinParams best = h->bp;
    float best_ms = 0;
    int trials = 0;
    try {
        best_ms = autotune_trial(h, s, best, sample, I, J, O, e0, e1);
        ++trials;
        for (const Knob& kb : knobs) {
            const int32_t start = best.*kb.field;
            for (int32_t v : kb.values) {
                if (v == start || trials >= max_trials) continue;
                BinParams cand = best;
                cand.*kb.field = v;
                float ms = 0;
                ++trials;
                try {
                    ms = autotune_trial(h, s, cand, sample, I, J, O, e0, e1);
                } catch (const Error& e) {
                    // a binning this graph cannot take (too many items, no memory)
                    if (e.code != SLG_ECAPACITY && e.code != SLG_ENOMEM) throw;
                    continue;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best = cand;
                }
            }
        }
    } catch (...) {
        h->plan.release(h->st);
        dfree(buf, h->st);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    h->plan.release(h->st);
    dfree(buf, h->st);
    SLG_CUDA_TRY(cudaEventDestroy(e0));
    SLG_CUDA_TRY(cudaEventDestroy(e1));
    h->bp = best;
    if (best_ms_out) *best_ms_out = best_ms;
}

}  // namespace slg
