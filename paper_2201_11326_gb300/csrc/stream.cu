// One-walk windows: the canonical lists of L_s(H) (and of an ensemble) window
// by window, each sparse-accumulator and hub-pair row walked once.
//
// Algorithm 2 (Section III-C) counts a row's pairs and writes them from one
// pass over its wedges; the count-then-fill form used elsewhere walks every row
// twice because the row offsets of the whole list must be known before a
// window is placed. Here a window's rows are chosen before their walk, from an
// upper bound on their pairs, so only the window's own offsets are needed:
//   * before the first window, the rows of the cheap handlers (tables, dense)
//     are counted exactly; a sparse-accumulator row i has at most W_i / s pairs
//     (every pair with overlap >= s takes s of its wedges) and a hub-pair row at
//     most Wp_i / (s - 1) (a partner sharing u non-hub vertices and t hubs,
//     u + t >= s, is met u + t(t-1)/2 >= s - 1 times among the walked entries);
//   * a window takes the rows whose bound, scaled by what the windows before it
//     observed (pairs per unit of bound; pairs of every list per list-0 pair),
//     fills nine tenths of the buffer;
//   * its sparse-accumulator and hub-pair items run their fill kernels as the
//     counting pass, staging each item's pairs and count (the staged counting
//     pass); the window's offsets are a scan of its items' counts; the fill
//     copies staged items into place and walks only the others (other handlers,
//     and items the pool could not hold);
//   * when the rows' list 0 exceeds the buffer after all, the window ends at the
//     last row that fits (the staged pairs of the rows after it are dropped and
//     those rows start the next window);
//   * in an ensemble (Algorithm 3) list t of the window is list t-1 filtered by
//     s_t (the lists are nested and in the same order); when they do not fit,
//     the window's rows are halved until they do.
#include <algorithm>

#include "handle.cuh"

namespace slg {
namespace {

int grid_of(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

// Upper bound on row i's pairs at threshold s0 before its walk (above).
__global__ void k_stream_bound(const int32_t* __restrict__ row_item,
                               const Item* __restrict__ items, const int64_t* __restrict__ W,
                               const int64_t* __restrict__ Wp, const int32_t* __restrict__ icnt,
                               int32_t s0, int32_t m, int64_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q0 = row_item[i], q1 = row_item[i + 1];
        int64_t b = 0;
        if (q1 > q0) {
            const int mode = items[q0].mode;
            if (mode == MODE_SPARSE) {
                b = W[i] / (s0 > 1 ? s0 : 1);
            } else if (mode == MODE_HUBPAIR) {
                const int64_t w = Wp ? Wp[i] : W[i];
                b = (w > 0 ? w : 0) / (s0 > 2 ? s0 - 1 : 1);
            } else {
                for (int32_t q = q0; q < q1; ++q) b += icnt[q];
            }
        }
        const int64_t later = (int64_t)m - 1 - i;  // partners j > i
        out[i] = b < later ? b : later;
    }
}

// rowoff[r] = ioff[row_item[r]] for r in [r0, r1]
__global__ void k_rowoff_range(const int32_t* __restrict__ row_item,
                               const int64_t* __restrict__ ioff, int32_t r0, int32_t r1,
                               int64_t* __restrict__ rowoff) {
    for (int64_t r = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= r1;
         r += (int64_t)gridDim.x * blockDim.x)
        rowoff[r] = ioff[row_item[r]];
}

// The largest r in [lo, hi] with cum[r] - cum[lo] <= budget (cum ascending).
__global__ void k_last_within(const int64_t* __restrict__ cum, int32_t lo, int32_t hi,
                              int64_t budget, int32_t* __restrict__ out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int64_t base = cum[lo];
    int32_t a = lo, b = hi;  // cum[a] - base <= budget; the answer lies in [a, b]
    while (a < b) {
        const int32_t mid = a + (int32_t)(((int64_t)b - a + 1) / 2);
        if (cum[mid] - base <= budget)
            a = mid;
        else
            b = mid - 1;
    }
    *out = a;
}

template <typename T>
T read_one(const T* src, cudaStream_t st) {
    T v{};
    SLG_CUDA_TRY(cudaMemcpyAsync(&v, src, sizeof(T), cudaMemcpyDeviceToHost, st));
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    return v;
}

int32_t last_within(const int64_t* cum, int32_t lo, int32_t hi, int64_t budget, cudaStream_t st) {
    int32_t* d = dalloc<int32_t>(1, st);
    k_last_within<<<1, 32, 0, st>>>(cum, lo, hi, budget, d);
    SLG_LAUNCH_CHECK();
    const int32_t r = read_one(d, st);
    dfree(d, st);
    return r;
}

// The plan for s[0], the exact counts of the rows that are not staged and
// the cumulative row bounds.
void stream_prepare(slg_graph* h, const int32_t* s, int32_t k) {
    Plan& p = h->plan;
    if (!(p.built && p.s == s[0])) build_plan(h, s[0], h->bp);
    p.release_ensemble(h->st);
    p.release_stream(h->st);
    p.counted = false;
    p.stage_s = -1;
    const int32_t m = h->g.m;
    constexpr unsigned STAGED = (1u << MODE_SPARSE) | (1u << MODE_HUBPAIR);
    run_count_modes(h->g, p, p.rs, ~STAGED, p.icnt, &h->mtimer, h->st);
    int64_t* b = dalloc<int64_t>((size_t)m + 1, h->st);
    p.stream_cum = dalloc<int64_t>((size_t)m + 1, h->st);
    if (m) {
        k_stream_bound<<<grid_of(m, 256), 256, 0, h->st>>>(p.row_item, p.items, p.W, p.Wp, p.icnt,
                                                          s[0], m, b);
        SLG_LAUNCH_CHECK();
    }
    scan_i64_to_i64(b, p.stream_cum, m, h->st);
    dfree(b, h->st);
    p.stream_k = k;
    std::copy(s, s + k, p.stream_s);
    p.stream_lambda = 1.0;
    p.stream_phi = (double)k;  // until a window has shown the later lists' share
}

// A pool for windows of cap pairs (cap plus a chunk per CTA, within the
// memory budget), kept while the windows' chunk size stays the same.
void stream_pool(slg_graph* h, int64_t cap) {
    Plan& p = h->plan;
    const int64_t ctas = 1024;
    const int64_t chunk = std::max<int64_t>(4096, std::min<int64_t>(SG_CHUNK, cap / (4 * ctas)));
    const int64_t want = cap + (ctas + 16) * chunk;
    if (p.stage_at && p.stage_cap > 0 && p.stage_chunk == chunk) return;
    p.release_stage(h->st);
    if (!can_stage(h)) return;
    alloc_stage(h, want, chunk);
}

}  // namespace

void stream_window(slg_graph* h, const int32_t* s, int32_t k, int32_t r0, int32_t* I,
                   int32_t* J, int32_t* O, int64_t cap, int32_t* r1_out, int64_t* pairs) {
    Plan& p = h->plan;
    const int32_t m = h->g.m;
    if (!(p.built && p.s == s[0] && p.stream_cum && p.stream_k == k &&
          std::equal(s, s + k, p.stream_s)))
        stream_prepare(h, s, k);
    for (int32_t t = 0; t < k; ++t) pairs[t] = 0;
    if (r0 >= m) {
        *r1_out = m;
        return;
    }
    p.counted = false;  // the plan's offsets now hold windows
    p.stage_s = -1;
    stream_pool(h, cap);
    cudaStream_t st = h->st;

    // rows whose scaled bound fills nine tenths of the buffer (one row at least)
    const double scale = std::max(p.stream_lambda * p.stream_phi, 1e-9);
    const double target = std::min(0.9 * (double)cap / scale, 9.0e18);
    int32_t r1 = last_within(p.stream_cum, r0, m, (int64_t)target, st);
    if (r1 <= r0) r1 = r0 + 1;
    const int32_t q0 = read_one(p.row_item + r0, st);
    int32_t q1 = read_one(p.row_item + r1, st);

    // list 0: counting (and staging) of the window's sparse-accumulator and
    // hub-pair items, then the window's offsets
    run_count_staged(h->g, p, p.rs, q0, q1, p.icnt, &h->mtimer, st);
    if (q1 > q0) scan_i32_to_i64(p.icnt + q0, p.ioff + q0, q1 - q0, st);
    else SLG_CUDA_TRY(cudaMemsetAsync(p.ioff + q0, 0, sizeof(int64_t), st));
    k_rowoff_range<<<grid_of((int64_t)r1 - r0 + 1, 256), 256, 0, st>>>(p.row_item, p.ioff, r0,
                                                                      r1, p.rowoff);
    SLG_LAUNCH_CHECK();
    int64_t P0 = read_one(p.rowoff + r1, st);
    if (P0 > cap) {  // the rows whose list 0 fits
        r1 = last_within(p.rowoff, r0, r1, cap, st);
        if (r1 <= r0) throw Error{SLG_ECAPACITY, "a single row has more pairs than cap"};
        q1 = read_one(p.row_item + r1, st);
        P0 = read_one(p.rowoff + r1, st);
    }
    StageUse su;
    if (p.stage_at && p.stage_cap > 0) su.st_ioff = p.ioff;
    run_fill(h->g, p, p.rs, p.ioff, q0, q1, I, J, O, P0, &h->mtimer, st, su);

    // the later lists, each filtered from the one before (timed while timing is on)
    int64_t seg[ENS_MAX + 1];
    seg[0] = 0;
    seg[1] = P0;
    int64_t fus[ENS_MAX] = {};
    for (;;) {
        bool fits = true;
        for (int32_t t = 1; t < k && fits; ++t) {
            const int64_t n = seg[t] - seg[t - 1], room = cap - seg[t];
            if (h->mtimer.on) SLG_CUDA_TRY(cudaEventRecord(h->mtimer.fev[0], st));
            const int64_t got = run_filter_room(I + seg[t - 1], J + seg[t - 1], O + seg[t - 1], n,
                                                s[t], I + seg[t], J + seg[t], O + seg[t], room, st);
            if (h->mtimer.on) {
                float ms = 0;
                SLG_CUDA_TRY(cudaEventRecord(h->mtimer.fev[1], st));
                SLG_CUDA_TRY(cudaEventSynchronize(h->mtimer.fev[1]));
                SLG_CUDA_TRY(cudaEventElapsedTime(&ms, h->mtimer.fev[0], h->mtimer.fev[1]));
                fus[t] += (int64_t)(1000.0f * ms);
            }
            if (got > room) fits = false;
            else seg[t + 1] = seg[t] + got;
        }
        if (fits) break;
        // halve the window's rows: list 0 of the first rows is a prefix of the
        // list in place
        const int32_t rh = r0 + (r1 - r0) / 2;
        if (rh <= r0) throw Error{SLG_ECAPACITY, "a single row's lists have more pairs than cap"};
        r1 = rh;
        seg[1] = read_one(p.rowoff + r1, st);
    }
    for (int32_t t = 0; t < k; ++t) {
        pairs[t] = seg[t + 1] - seg[t];
        int64_t* mk = h->ens_made[t];  // slg_ensemble_fill_stats
        mk[t == 0 ? 0 : 2] += 1;
        mk[t == 0 ? 1 : 3] += pairs[t];
        mk[4] += fus[t];
        if (t > 0) mk[5] += seg[t] - seg[t - 1];
    }
    const int64_t bound = read_one(p.stream_cum + r1, st) - read_one(p.stream_cum + r0, st);
    if (bound > 0 && seg[1] > 0) p.stream_lambda = (double)seg[1] / (double)bound;
    if (seg[1] > 0) p.stream_phi = (double)seg[k] / (double)seg[1];
    *r1_out = r1;
}

}  // namespace slg
