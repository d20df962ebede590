// C-ABI entry points of libslg (declared in include/slg.h).
//
// Host orchestration only: every step of the computation runs in the kernels
// of transpose.cu, plan.cu, count_fill.cu and scan.cu. There is no CPU path.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <vector>

#include "handle.cuh"

namespace slg {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};
static std::atomic<long long> g_stage_bytes{0};  // staging pools held by all handles

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void stage_bytes_add(int64_t d) { g_stage_bytes.fetch_add(d, std::memory_order_relaxed); }

void set_error(slg_status code, const std::string& msg) {
    (void)code;
    g_last_error = msg;
}

namespace {

__global__ void k_size_range(const int32_t* __restrict__ size, int32_t m,
                             int32_t* __restrict__ mm) {
    int32_t lo = INT32_MAX, hi = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t z = size[i];
        if (z > 0) lo = min(lo, z);
        hi = max(hi, z);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&mm[0], lo);
        atomicMax(&mm[1], hi);
    }
}

}  // namespace

// Device memory the kernels may write: managed memory, or device memory of
// the current device. Device memory of another GPU is refused (an error, not
// a host copy: the kernels cannot reach it without a peer mapping).
bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    if (a.type != cudaMemoryTypeDevice) return false;
    int dev = -1;
    SLG_CUDA_TRY(cudaGetDevice(&dev));
    if (a.device != dev)
        throw Error{SLG_EINVAL, "an array lies in another GPU's memory than the current device's"};
    return true;
}

namespace {


}  // namespace

BinParams default_bins() {
    BinParams b;
    b.warp_max_wedges = 128;
    b.block_item_wedges = 1024;
    b.dense_min_density = 64;  // dense when W_i >= span / 4
    b.dense_item_tiles = 4;
    b.wdense_max_ranges = WD_MAXR;
    b.sparse_min_per_tile = 64;
    b.sparse_item_wedges = 65536;
    b.wsparse_max_size = WS_MAXE;
    return b;
}

void Timer::init() {
    for (auto& e : ev)
        if (!e) SLG_CUDA_TRY(cudaEventCreate(&e));
}
void Timer::mark(int k, cudaStream_t st) {
    if (on) SLG_CUDA_TRY(cudaEventRecord(ev[k], st));
}
void Timer::destroy() {
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
}

void mtimer_init(ModeTimer& t) {
    for (auto& e : t.ev)
        if (!e) SLG_CUDA_TRY(cudaEventCreate(&e));
    for (auto& e : t.fev)
        if (!e) SLG_CUDA_TRY(cudaEventCreate(&e));
}

void build_plan(slg_graph* h, int32_t s, const BinParams& bp) {
    Plan& p = h->plan;
    const bool allowed = s >= 2 && h->owns_data && !h->g.srow && h->hp_max_hubs >= 2;
    if (!allowed) {
        plan_build(h->g, s, bp, p, h->st, nullptr);
        return;
    }
    if (!h->hp.built && !h->hp.tried) {
        // decide on the plan without hub pairs: worth it only when the rows that
        // would walk every wedge (table and sparse-accumulator rows) carry many
        plan_build(h->g, s, bp, p, h->st, nullptr);
        const int64_t sw = plan_sparse_wedges(h->g, p, h->st);
        if (sw == 0 || sw < h->hp_min_wedges) return;
        hubpair_build(h->g, std::min(h->hp_max_hubs, HP_MAXK), h->hp_max_pairs, h->hp, h->st);
        if (!h->hp.built) return;
    }
    plan_build(h->g, s, bp, p, h->st, h->hp.built ? &h->hp : nullptr);
}

// A staging pool (StageArgs) of at most `want` pairs in chunks of `chunk`:
// three quarters of the free device memory beyond 6 GiB, at most
// stage_max_bytes when set (else all handles' pools under a quarter of the
// device's memory), at most 2^34 pairs. False (and no pool) when fewer than 16
// chunks (automatic) or one chunk (capped) fit.
bool alloc_stage(slg_graph* h, int64_t want, int64_t chunk) {
    Plan& p = h->plan;
    SLG_CUDA_TRY(cudaStreamSynchronize(h->st));  // released buffers are back with the device
    size_t fr = 0, tot = 0;
    SLG_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    int64_t budget = ((int64_t)fr - ((int64_t)6 << 30)) / 4 * 3;
    if (h->stage_max_bytes > 0) budget = std::min(budget, h->stage_max_bytes);
    else budget = std::min(budget, (int64_t)(tot / 4) - (int64_t)g_stage_bytes.load());
    int64_t cap = std::min<int64_t>((budget - 8 * p.nitems) / 5, (int64_t)1 << 34);
    cap = std::min(cap, want);
    if (cap < (h->stage_max_bytes > 0 ? chunk : 16 * chunk)) return false;
    p.stage_chunk = chunk;
    p.stage_at = dalloc<int64_t>((size_t)p.nitems, h->st);
    p.stage_J = dalloc<int32_t>((size_t)cap, h->st);
    p.stage_O = dalloc<uint8_t>((size_t)cap, h->st);
    p.stage_cursor = dalloc<unsigned long long>(1, h->st);
    p.stage_cap = cap;
    p.stage_bytes = 8 * p.nitems + 5 * cap;
    stage_bytes_add(p.stage_bytes);
    return true;
}

bool can_stage(const slg_graph* h) {
    const Plan& p = h->plan;
    if (h->stage_max_bytes == 0 || !h->owns_data) return false;
    return p.mode_count[MODE_SPARSE] > 0 || (p.mode_count[MODE_HUBPAIR] > 0 && p.hp);
}

// The counting pass's staging pool for a plan with sparse-accumulator or
// hub-pair items: no more than those rows can fill (their walk, plus a chunk
// per CTA). The pool lives as long as the plan, so the automatic one is only
// made when the rows can fill at least 2^26 pairs (a second walk of fewer costs
// little). Views (which share their device with other queries) stage nothing.
void plan_staging(slg_graph* h) {
    Plan& p = h->plan;
    p.release_stage(h->st);
    if (!can_stage(h)) return;
    // chunks: a CTA's share of what the rows can fill, between 2^12 and 2^20 pairs
    const int64_t bound = plan_stage_bound(h->g, p, h->st);
    if (h->stage_max_bytes < 0 && bound < ((int64_t)1 << 26)) return;
    const int64_t ctas = 1024;  // CTAs of the two handlers' fill launches, about
    const int64_t chunk = std::max<int64_t>(4096, std::min<int64_t>(SG_CHUNK, bound / (4 * ctas)));
    alloc_stage(h, bound + (ctas + 16) * chunk, chunk);
}

slg_graph* make_view(const slg_graph* base, cudaStream_t st) {
    slg_graph* h = new slg_graph();
    h->g = base->g;
    h->owns_data = false;
    h->st = st;
    h->device = base->device;
    h->bp = base->bp;
    try {
        h->timer.init();
        mtimer_init(h->mtimer);
    } catch (...) {
        delete h;
        throw;
    }
    return h;
}

}  // namespace slg

using slg::Error;

namespace {

slg_status fail(slg_status code, const std::string& msg) {
    slg::set_error(code, msg);
    return code;
}

#define API_BEGIN try {
#define API_END                                              \
    }                                                        \
    catch (const Error& e) {                                 \
        return fail(e.code, e.msg);                          \
    }                                                        \
    catch (const std::exception& e) {                        \
        return fail(SLG_EINTERNAL, e.what());                \
    }                                                        \
    slg::g_last_error.clear();                               \
    return SLG_OK;

void free_graph_dev(slg::GraphDev& g, cudaStream_t st) {
    slg::dfree(g.off, st);
    slg::dfree(g.idx, st);
    slg::dfree(g.size, st);
    slg::dfree(g.rowid, st);
    slg::dfree(g.offT, st);
    slg::dfree(g.idxT, st);
    slg::dfree(g.tpos, st);
    slg::dfree(g.hubidx, st);
    slg::dfree(g.hubmask, st);
    slg::dfree(g.srow, st);
    slg::dfree(g.rbase, st);
}

// Count pass for s (cached per handle): plan, count, offsets.
void check_s(const slg_graph* h, int32_t s) {
    if (h->g.srow) {
        if (s != 0) throw Error{SLG_EINVAL, "a batch uses each graph's own s: pass s = 0"};
    } else if (s < 1) {
        throw Error{SLG_EINVAL, "s must be >= 1"};
    }
}

void ensure_counted(slg_graph* h, int32_t s) {
    check_s(h, s);
    slg::Plan& p = h->plan;
    if (p.built && p.s == s && p.counted) return;
    h->timer.mark(0, h->st);
    if (!(p.built && p.s == s)) slg::build_plan(h, s, h->bp);
    slg::plan_staging(h);
    p.stage_s = s;
    h->timer.mark(1, h->st);
    slg::run_count(h->g, p, p.rs, p.icnt, &h->mtimer, h->st);
    h->timer.mark(2, h->st);
    slg::plan_offsets(h->g, p, h->st);  // synchronises
    h->timer.mark(3, h->st);
    if (h->timer.on) {
        SLG_CUDA_TRY(cudaEventSynchronize(h->timer.ev[3]));
        SLG_CUDA_TRY(cudaEventElapsedTime(&h->ms[0], h->timer.ev[0], h->timer.ev[1]));
        SLG_CUDA_TRY(cudaEventElapsedTime(&h->ms[1], h->timer.ev[1], h->timer.ev[2]));
        SLG_CUDA_TRY(cudaEventElapsedTime(&h->ms[2], h->timer.ev[2], h->timer.ev[3]));
        h->ms[3] = h->ms[4] = 0;
    }
}

// Ensemble for s_list (Algorithm 3): the plan built for s_list[0], every
// list counted (cached per handle, like ensure_counted).
void check_s_list(const slg_graph* h, const int32_t* s_list, int32_t k) {
    if (h->g.srow) throw Error{SLG_EINVAL, "an ensemble takes one graph, not a batch"};
    if (!s_list || k < 1 || k > slg::ENS_MAX)
        throw Error{SLG_EINVAL, "an ensemble takes 1 to 16 thresholds"};
    for (int32_t t = 0; t < k; ++t) {
        if (s_list[t] < 1) throw Error{SLG_EINVAL, "s must be >= 1"};
        if (t > 0 && s_list[t] <= s_list[t - 1])
            throw Error{SLG_EINVAL, "ensemble thresholds must be strictly ascending"};
    }
}

void ensure_ensemble(slg_graph* h, const int32_t* s_list, int32_t k) {
    check_s_list(h, s_list, k);
    slg::Plan& p = h->plan;
    if (p.built && p.s == s_list[0] && p.ens.counted && p.ens.k == k &&
        std::equal(s_list, s_list + k, p.ens.s))
        return;
    h->timer.mark(0, h->st);
    if (!(p.built && p.s == s_list[0])) slg::build_plan(h, s_list[0], h->bp);
    h->timer.mark(1, h->st);
    slg::ensemble_count(h->g, p, s_list, k, &h->mtimer, h->st);  // synchronises
    h->timer.mark(2, h->st);
    h->timer.mark(3, h->st);
    if (h->timer.on) {
        SLG_CUDA_TRY(cudaEventSynchronize(h->timer.ev[3]));
        SLG_CUDA_TRY(cudaEventElapsedTime(&h->ms[0], h->timer.ev[0], h->timer.ev[1]));
        SLG_CUDA_TRY(cudaEventElapsedTime(&h->ms[1], h->timer.ev[1], h->timer.ev[2]));
        h->ms[2] = h->ms[3] = h->ms[4] = 0;
    }
}

// Copy `bytes` from device src to dst (host or device).
void copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (bytes) SLG_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
}

struct WindowInfo {
    int64_t base, end;
    int32_t q0, q1;
};

WindowInfo window_info(slg_graph* h, int32_t r0, int32_t r1) {
    WindowInfo w;
    SLG_CUDA_TRY(cudaMemcpyAsync(&w.base, h->plan.rowoff + r0, 8, cudaMemcpyDeviceToHost, h->st));
    SLG_CUDA_TRY(cudaMemcpyAsync(&w.end, h->plan.rowoff + r1, 8, cudaMemcpyDeviceToHost, h->st));
    SLG_CUDA_TRY(cudaMemcpyAsync(&w.q0, h->plan.row_item + r0, 4, cudaMemcpyDeviceToHost, h->st));
    SLG_CUDA_TRY(cudaMemcpyAsync(&w.q1, h->plan.row_item + r1, 4, cudaMemcpyDeviceToHost, h->st));
    SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
    return w;
}

// Fill rows [r0, r1) into device buffers I/J/O (at least end-base entries),
// optionally digesting. Returns the pair count.
int64_t fill_window_dev(slg_graph* h, int32_t r0, int32_t r1, int32_t* I, int32_t* J,
                        int32_t* O, unsigned long long* dtot, unsigned long long* drows,
                        const WindowInfo& w) {
    const int64_t P = w.end - w.base;
    h->timer.mark(3, h->st);
    const slg::Plan& p = h->plan;
    slg::StageUse su;
    if (p.stage_s == p.s) su.st_ioff = p.ioff;  // this list was staged
    slg::run_fill(h->g, p, p.rs, p.ioff, w.q0, w.q1, I, J, O, P, &h->mtimer, h->st, su);
    h->timer.mark(4, h->st);
    if (dtot || drows)
        slg::run_digest(h->plan.rs, h->plan.rowoff, r0, r1, I, J, O, P, dtot, drows, h->st);
    h->timer.mark(5, h->st);
    return P;
}

void finish_timing(slg_graph* h, int64_t pairs_written) {
    if (!h->timer.on) return;
    SLG_CUDA_TRY(cudaEventSynchronize(h->timer.ev[5]));
    SLG_CUDA_TRY(cudaEventElapsedTime(&h->ms[3], h->timer.ev[3], h->timer.ev[4]));
    SLG_CUDA_TRY(cudaEventElapsedTime(&h->ms[4], h->timer.ev[4], h->timer.ev[5]));
    (void)pairs_written;
}

}  // namespace

extern "C" {

const char* slg_last_error(void) { return slg::g_last_error.c_str(); }

int32_t slg_version(void) { return 100; }

slg_status slg_load(const int32_t* off, const int32_t* idx, int32_t m, int32_t n, void* stream,
                    slg_graph** out) {
    if (!out) return fail(SLG_EINVAL, "out is NULL");
    *out = nullptr;
    if (m < 0 || n < 0) return fail(SLG_EINVAL, "m and n must be >= 0");
    if (!off) return fail(SLG_EINVAL, "off is NULL");
    slg_graph* h = new slg_graph();
    h->st = (cudaStream_t)stream;
    try {
        SLG_CUDA_TRY(cudaGetDevice(&h->device));
        slg::GraphDev& g = h->g;
        g.m = m;
        g.n = n;
        int32_t off_m = 0, off_0 = 0;
        copy_out(&off_m, off + m, sizeof(int32_t), h->st);
        copy_out(&off_0, off, sizeof(int32_t), h->st);
        SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
        if (off_0 != 0 || off_m < 0) throw Error{SLG_EINVAL, "off[0] must be 0 and off[m] >= 0"};
        g.nnz = off_m;
        if (g.nnz > 0 && !idx) throw Error{SLG_EINVAL, "idx is NULL"};
        g.off = slg::dalloc<int32_t>((size_t)m + 1, h->st);
        g.idx = slg::dalloc<int32_t>((size_t)g.nnz + 4, h->st);
        g.size = slg::dalloc<int32_t>((size_t)m, h->st);
        g.rowid = slg::dalloc<int32_t>((size_t)g.nnz + 4, h->st);
        g.offT = slg::dalloc<int32_t>((size_t)n + 1, h->st);
        g.idxT = slg::dalloc<int32_t>((size_t)g.nnz + 4, h->st);
        g.tpos = slg::dalloc<int32_t>((size_t)g.nnz + 4, h->st);
        copy_out(g.off, off, sizeof(int32_t) * ((size_t)m + 1), h->st);
        copy_out(g.idx, idx, sizeof(int32_t) * (size_t)g.nnz, h->st);
        SLG_CUDA_TRY(cudaMemsetAsync(g.rowid, 0, sizeof(int32_t) * ((size_t)g.nnz + 4), h->st));
        SLG_CUDA_TRY(cudaMemsetAsync(g.idxT + g.nnz, 0, sizeof(int32_t) * 4, h->st));
        int32_t* flag = slg::dalloc<int32_t>(3, h->st);
        slg::launch_validate(g.off, g.idx, m, n, g.nnz, g.rowid, g.size, flag, h->st);
        int32_t mm_init[2] = {INT32_MAX, 0};
        SLG_CUDA_TRY(cudaMemcpyAsync(flag + 1, mm_init, sizeof(mm_init), cudaMemcpyHostToDevice,
                                     h->st));
        if (m) {
            slg::k_size_range<<<152 * 4, 256, 0, h->st>>>(g.size, m, flag + 1);
            SLG_LAUNCH_CHECK();
        }
        int32_t fl[3];
        SLG_CUDA_TRY(cudaMemcpyAsync(fl, flag, sizeof(fl), cudaMemcpyDeviceToHost, h->st));
        SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
        slg::dfree(flag, h->st);
        if (fl[0]) {
            char buf[160];
            snprintf(buf, sizeof(buf), "invalid CSR:%s%s%s",
                     (fl[0] & 1) ? " offsets not monotone or out of range;" : "",
                     (fl[0] & 2) ? " vertex id outside [0, n);" : "",
                     (fl[0] & 4) ? " row not strictly increasing (repeated or unsorted vertex);"
                                 : "");
            throw Error{SLG_EINVAL, buf};
        }
        g.min_size = fl[1] == INT32_MAX ? 0 : fl[1];
        g.max_size = fl[2];
        slg::build_transpose(g.idx, g.rowid, n, g.nnz, g.offT, g.idxT, g.tpos, h->st);
        g.hubidx = slg::dalloc<int32_t>((size_t)n + 1, h->st);
        // +64: the warp dense handler reads hub masks 4 at a time from 32-aligned tiles
        g.hubmask = slg::dalloc<uint32_t>((size_t)m + 64, h->st);
        SLG_CUDA_TRY(cudaMemsetAsync(g.hubmask, 0, sizeof(uint32_t) * ((size_t)m + 64), h->st));
        g.nhubs = slg::build_hubs(g.off, g.idx, g.offT, m, n, g.hubidx, g.hubmask, h->st);
        SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
        h->timer.init();
        slg::mtimer_init(h->mtimer);
    } catch (const Error& e) {
        h->plan.release(h->st);
        free_graph_dev(h->g, h->st);
        cudaStreamSynchronize(h->st);
        delete h;
        return fail(e.code, e.msg);
    }
    *out = h;
    slg::g_last_error.clear();
    return SLG_OK;
}

void slg_free(slg_graph* h) {
    if (!h) return;
    try {
        h->plan.release(h->st);
    } catch (...) {
    }
    if (h->owns_data) free_graph_dev(h->g, h->st);
    h->hp.release(h->st);
    cudaStreamSynchronize(h->st);
    h->timer.destroy();
    for (auto& e : h->mtimer.ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : h->mtimer.fev)
        if (e) cudaEventDestroy(e);
    delete h;
}

slg_status slg_graph_info(const slg_graph* h, int32_t* m, int32_t* n, int64_t* nnz) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    if (m) *m = h->g.m;
    if (n) *n = h->g.n;
    if (nnz) *nnz = h->g.nnz;
    return SLG_OK;
}

slg_status slg_transpose_copy(slg_graph* h, int32_t* offT, int32_t* idxT) {
    if (!h || !offT || (!idxT && h->g.nnz)) return fail(SLG_EINVAL, "NULL argument");
    API_BEGIN
    copy_out(offT, h->g.offT, sizeof(int32_t) * ((size_t)h->g.n + 1), h->st);
    copy_out(idxT, h->g.idxT, sizeof(int32_t) * (size_t)h->g.nnz, h->st);
    SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
    API_END
}

slg_status slg_count(slg_graph* h, int32_t s, int64_t* pairs, int64_t* wedges) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    API_BEGIN
    ensure_counted(h, s);
    if (pairs) *pairs = h->plan.pairs;
    if (wedges) *wedges = h->plan.wedges;
    API_END
}

slg_status slg_bound(slg_graph* h, int32_t s, int64_t* pairs_ub) {
    if (!h || !pairs_ub) return fail(SLG_EINVAL, "NULL argument");
    API_BEGIN
    check_s(h, s);
    if (!h->plan.built || h->plan.s != s) slg::build_plan(h, s, h->bp);
    // every s-incident pair accounts for at least s wedges (at least 1 in a batch)
    *pairs_ub = h->plan.wedges / (s > 0 ? s : 1);
    API_END
}

slg_status slg_row_offsets(slg_graph* h, int32_t s, int64_t* rowoff) {
    if (!h || !rowoff) return fail(SLG_EINVAL, "NULL argument");
    API_BEGIN
    ensure_counted(h, s);
    copy_out(rowoff, h->plan.rowoff, sizeof(int64_t) * ((size_t)h->g.m + 1), h->st);
    SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
    API_END
}

slg_status slg_build_window(slg_graph* h, int32_t s, int32_t r0, int32_t r1, int32_t* I,
                            int32_t* J, int32_t* O, int64_t cap, int64_t* pairs,
                            uint64_t* digest, uint64_t* row_digests) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    if (r0 < 0 || r1 < r0 || r1 > h->g.m) return fail(SLG_EINVAL, "bad row range");
    API_BEGIN
    ensure_counted(h, s);
    const WindowInfo w = window_info(h, r0, r1);
    const int64_t P = w.end - w.base;
    if (pairs) *pairs = P;
    if (P > cap) throw Error{SLG_ECAPACITY, "output buffer too small for the window"};
    if (P > 0 && (!I || !J || !O)) throw Error{SLG_EINVAL, "NULL output array"};
    const bool dev = P == 0 || (slg::is_device_ptr(I) && slg::is_device_ptr(J) && slg::is_device_ptr(O));
    int32_t *dI = I, *dJ = J, *dO = O;
    if (!dev) {
        dI = slg::dalloc<int32_t>(P, h->st);
        dJ = slg::dalloc<int32_t>(P, h->st);
        dO = slg::dalloc<int32_t>(P, h->st);
    }
    unsigned long long* dd = nullptr;
    const int32_t nr = r1 - r0;
    if (digest || row_digests) {
        dd = slg::dalloc<unsigned long long>((size_t)nr + 1, h->st);
        SLG_CUDA_TRY(cudaMemsetAsync(dd, 0, sizeof(unsigned long long) * ((size_t)nr + 1), h->st));
    }
    fill_window_dev(h, r0, r1, dI, dJ, dO, dd, row_digests ? dd + 1 : nullptr, w);
    if (!dev) {
        copy_out(I, dI, sizeof(int32_t) * P, h->st);
        copy_out(J, dJ, sizeof(int32_t) * P, h->st);
        copy_out(O, dO, sizeof(int32_t) * P, h->st);
    }
    if (digest) copy_out(digest, dd, sizeof(uint64_t), h->st);
    if (row_digests) copy_out(row_digests, dd + 1, sizeof(uint64_t) * nr, h->st);
    SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
    finish_timing(h, P);
    if (!dev) {
        slg::dfree(dI, h->st);
        slg::dfree(dJ, h->st);
        slg::dfree(dO, h->st);
    }
    slg::dfree(dd, h->st);
    API_END
}

slg_status slg_build(slg_graph* h, int32_t s, int32_t* I, int32_t* J, int32_t* O, int64_t cap,
                     int64_t* pairs) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    API_BEGIN
    ensure_counted(h, s);
    const int64_t P = h->plan.pairs;
    if (pairs) *pairs = P;
    if (P > cap) throw Error{SLG_ECAPACITY, "output buffer too small"};
    if (P == 0) {
        slg::g_last_error.clear();
        return SLG_OK;
    }
    if (!I || !J || !O) throw Error{SLG_EINVAL, "NULL output array"};
    const bool dev = slg::is_device_ptr(I) && slg::is_device_ptr(J) && slg::is_device_ptr(O);
    if (dev) {
        WindowInfo w{0, P, 0, (int32_t)h->plan.nitems};
        fill_window_dev(h, 0, h->g.m, I, J, O, nullptr, nullptr, w);
        SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
        finish_timing(h, P);
    } else {
        // host destination: produce bounded windows through a device staging buffer
        const int64_t stage = (int64_t)1 << 27;  // pairs per window (1.5 GiB staging)
        const int64_t maxrow = slg::plan_max_row(h->g, h->plan.rowoff, h->st);
        const int64_t cap_w = stage > maxrow ? stage : maxrow;
        const int64_t C = cap_w - maxrow > 0 ? cap_w - maxrow : 1;
        int32_t* splits_d = slg::dalloc<int32_t>((size_t)h->g.m + 1, h->st);
        const int32_t nw = slg::plan_windows(h->g, h->plan.rowoff, C, splits_d, h->st);
        std::vector<int32_t> splits((size_t)nw + 1);
        copy_out(splits.data(), splits_d, sizeof(int32_t) * nw, h->st);
        SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
        slg::dfree(splits_d, h->st);
        splits[nw] = h->g.m;
        int32_t* dI = slg::dalloc<int32_t>(cap_w, h->st);
        int32_t* dJ = slg::dalloc<int32_t>(cap_w, h->st);
        int32_t* dO = slg::dalloc<int32_t>(cap_w, h->st);
        for (int32_t k = 0; k < nw; ++k) {
            const WindowInfo w = window_info(h, splits[k], splits[k + 1]);
            const int64_t Pw = fill_window_dev(h, splits[k], splits[k + 1], dI, dJ, dO, nullptr,
                                               nullptr, w);
            copy_out(I + w.base, dI, sizeof(int32_t) * Pw, h->st);
            copy_out(J + w.base, dJ, sizeof(int32_t) * Pw, h->st);
            copy_out(O + w.base, dO, sizeof(int32_t) * Pw, h->st);
        }
        SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
        slg::dfree(dI, h->st);
        slg::dfree(dJ, h->st);
        slg::dfree(dO, h->st);
    }
    API_END
}

slg_status slg_plan_windows(slg_graph* h, int32_t s, int64_t cap, int32_t* row_splits,
                            int32_t max_windows, int32_t* nwindows) {
    if (!h || !row_splits || !nwindows) return fail(SLG_EINVAL, "NULL argument");
    if (cap < 1) return fail(SLG_EINVAL, "cap must be >= 1");
    API_BEGIN
    *nwindows = 0;
    ensure_counted(h, s);
    const int64_t maxrow = slg::plan_max_row(h->g, h->plan.rowoff, h->st);
    if (maxrow > cap) throw Error{SLG_ECAPACITY, "a single row has more pairs than cap"};
    const int64_t C = cap - maxrow > 0 ? cap - maxrow : 1;
    const int32_t nw = slg::plan_windows(h->g, h->plan.rowoff, C, nullptr, h->st);
    *nwindows = nw;
    if (nw > max_windows) throw Error{SLG_ECAPACITY, "more windows needed than max_windows"};
    int32_t* splits_d = slg::dalloc<int32_t>((size_t)nw + 1, h->st);
    slg::plan_windows(h->g, h->plan.rowoff, C, splits_d, h->st);
    copy_out(row_splits, splits_d, sizeof(int32_t) * nw, h->st);
    SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
    slg::dfree(splits_d, h->st);
    row_splits[nw] = h->g.m;
    API_END
}

slg_status slg_ensemble_count(slg_graph* h, const int32_t* s_list, int32_t k, int64_t* pairs,
                              int64_t* wedges) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    API_BEGIN
    ensure_ensemble(h, s_list, k);
    if (pairs)
        for (int32_t t = 0; t < k; ++t) pairs[t] = h->plan.ens.pairs[t];
    if (wedges) *wedges = h->plan.wedges;
    API_END
}

slg_status slg_ensemble_row_offsets(slg_graph* h, const int32_t* s_list, int32_t k,
                                    int64_t* rowoff) {
    if (!h || !rowoff) return fail(SLG_EINVAL, "NULL argument");
    API_BEGIN
    ensure_ensemble(h, s_list, k);
    copy_out(rowoff, h->plan.ens.rowoff, sizeof(int64_t) * (size_t)k * ((size_t)h->g.m + 1),
             h->st);
    SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
    API_END
}

slg_status slg_ensemble_plan_windows(slg_graph* h, const int32_t* s_list, int32_t k,
                                     int32_t which, int64_t cap, int32_t* row_splits,
                                     int32_t max_windows, int32_t* nwindows) {
    if (!h || !row_splits || !nwindows) return fail(SLG_EINVAL, "NULL argument");
    if (cap < 1) return fail(SLG_EINVAL, "cap must be >= 1");
    if (which < -1 || which >= k) return fail(SLG_EINVAL, "bad list selector");
    API_BEGIN
    *nwindows = 0;
    ensure_ensemble(h, s_list, k);
    const int64_t* tot = which < 0 ? h->plan.ens.rowtot
                                   : h->plan.ens.rowoff + (int64_t)which * ((int64_t)h->g.m + 1);
    const int64_t maxrow = slg::plan_max_row(h->g, tot, h->st);
    if (maxrow > cap) throw Error{SLG_ECAPACITY, "a single row has more pairs than cap"};
    const int64_t C = cap - maxrow > 0 ? cap - maxrow : 1;
    const int32_t nw = slg::plan_windows(h->g, tot, C, nullptr, h->st);
    *nwindows = nw;
    if (nw > max_windows) throw Error{SLG_ECAPACITY, "more windows needed than max_windows"};
    int32_t* splits_d = slg::dalloc<int32_t>((size_t)nw + 1, h->st);
    slg::plan_windows(h->g, tot, C, splits_d, h->st);
    copy_out(row_splits, splits_d, sizeof(int32_t) * nw, h->st);
    SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
    slg::dfree(splits_d, h->st);
    row_splits[nw] = h->g.m;
    API_END
}

slg_status slg_ensemble_build_window(slg_graph* h, const int32_t* s_list, int32_t k,
                                     int32_t which, int32_t r0, int32_t r1, int32_t* I,
                                     int32_t* J, int32_t* O, int64_t cap, int64_t* pairs,
                                     uint64_t* digests, uint64_t* row_digests) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    if (r0 < 0 || r1 < r0 || r1 > h->g.m) return fail(SLG_EINVAL, "bad row range");
    if (which < -1 || which >= k) return fail(SLG_EINVAL, "bad list selector");
    API_BEGIN
    ensure_ensemble(h, s_list, k);
    slg::Plan& p = h->plan;
    const int64_t m1 = (int64_t)h->g.m + 1, ni = p.nitems;
    // selected lists t0 .. t1-1; slice of each: rowoff_t[r0] .. rowoff_t[r1];
    // items row_item[r0] .. row_item[r1]
    const int32_t t0 = which < 0 ? 0 : which, t1 = which < 0 ? k : which + 1, nl = t1 - t0;
    int64_t base[slg::ENS_MAX], end[slg::ENS_MAX], seg[slg::ENS_MAX + 1];
    int32_t q0 = 0, q1 = 0;
    for (int32_t t = t0; t < t1; ++t) {
        copy_out(&base[t], p.ens.rowoff + t * m1 + r0, sizeof(int64_t), h->st);
        copy_out(&end[t], p.ens.rowoff + t * m1 + r1, sizeof(int64_t), h->st);
    }
    copy_out(&q0, p.row_item + r0, sizeof(int32_t), h->st);
    copy_out(&q1, p.row_item + r1, sizeof(int32_t), h->st);
    SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
    seg[0] = 0;  // seg is indexed by position among the selected lists
    for (int32_t t = t0; t < t1; ++t) {
        seg[t - t0 + 1] = seg[t - t0] + (end[t] - base[t]);
        if (pairs) pairs[t - t0] = end[t] - base[t];
    }
    const int64_t P = seg[nl];
    if (P > cap) throw Error{SLG_ECAPACITY, "output buffer too small for the window"};
    if (P > 0 && (!I || !J || !O)) throw Error{SLG_EINVAL, "NULL output array"};
    const bool dev = P == 0 || (slg::is_device_ptr(I) && slg::is_device_ptr(J) &&
                                slg::is_device_ptr(O));
    int32_t *dI = I, *dJ = J, *dO = O;
    if (!dev) {
        dI = slg::dalloc<int32_t>(P, h->st);
        dJ = slg::dalloc<int32_t>(P, h->st);
        dO = slg::dalloc<int32_t>(P, h->st);
    }
    const int32_t nr = r1 - r0;
    unsigned long long* dd = nullptr;  // per list: total, then one entry per row
    if (digests || row_digests) {
        const size_t nd = (size_t)nl * ((size_t)nr + 1);
        dd = slg::dalloc<unsigned long long>(nd, h->st);
        SLG_CUDA_TRY(cudaMemsetAsync(dd, 0, sizeof(unsigned long long) * nd, h->st));
    }
    h->timer.mark(3, h->st);
    // each selected list from the shared plan with its own threshold, into its
    // segment (one fused pass over all lists was measured slower: the lists
    // after the first went out as partial-line stores)
    // A list after the first in the window may instead be the list before it
    // filtered by its threshold (the lists are nested and in the same order):
    // that reads 16 bytes per pair of the list before (12 to copy, 4 to count), a
    // walk about 4 per entry it reads (wedges through vertices that are not mask
    // hubs; hub-pair rows' walked entries), so the filter is taken when
    // 6 * pairs < entries (or as slg_set_ensemble_filter says)
    int64_t wrows = -1;
    for (int32_t t = t0; t < t1; ++t) {
        const int32_t u = t - t0;
        bool filt = false;
        if (t > t0 && h->ens_filter != 0) {
            if (h->ens_filter > 0) {
                filt = true;
            } else {
                if (wrows < 0) wrows = slg::plan_row_walk(h->g, p, r0, r1, h->st);
                filt = 6 * (seg[u] - seg[u - 1]) < wrows;
            }
        }
        const bool ftimed = filt && h->mtimer.on;
        float fms = 0;
        if (ftimed) SLG_CUDA_TRY(cudaEventRecord(h->mtimer.fev[0], h->st));
        if (filt)
            slg::run_filter(dI + seg[u - 1], dJ + seg[u - 1], dO + seg[u - 1], seg[u] - seg[u - 1],
                            p.ens.s[t], dI + seg[u], dJ + seg[u], dO + seg[u], seg[u + 1] - seg[u],
                            h->st);
        if (ftimed) {
            SLG_CUDA_TRY(cudaEventRecord(h->mtimer.fev[1], h->st));
            SLG_CUDA_TRY(cudaEventSynchronize(h->mtimer.fev[1]));
            SLG_CUDA_TRY(cudaEventElapsedTime(&fms, h->mtimer.fev[0], h->mtimer.fev[1]));
        }
        if (!filt)
            slg::run_fill(h->g, p, p.rs_for(p.ens.s[t]), p.ens.ioff + t * (ni + 1), q0, q1,
                          dI + seg[u], dJ + seg[u], dO + seg[u], seg[u + 1] - seg[u], &h->mtimer,
                          h->st);
        if (t1 - t0 == k) {  // windows of every list
            int64_t* mk = h->ens_made[t];
            mk[filt ? 2 : 0] += 1;
            mk[filt ? 3 : 1] += seg[u + 1] - seg[u];
            mk[4] += (int64_t)(1000.0f * fms);
            if (filt) mk[5] += seg[u] - seg[u - 1];
        }
    }
    h->timer.mark(4, h->st);
    if (dd) {
        for (int32_t t = t0; t < t1; ++t) {
            const int32_t u = t - t0;
            unsigned long long* dt = dd + (size_t)u * ((size_t)nr + 1);
            slg::run_digest(p.rs_for(p.ens.s[t]), p.ens.rowoff + t * m1, r0, r1, dI + seg[u],
                            dJ + seg[u], dO + seg[u], seg[u + 1] - seg[u], dt,
                            row_digests ? dt + 1 : nullptr, h->st);
        }
    }
    h->timer.mark(5, h->st);
    if (!dev) {
        copy_out(I, dI, sizeof(int32_t) * P, h->st);
        copy_out(J, dJ, sizeof(int32_t) * P, h->st);
        copy_out(O, dO, sizeof(int32_t) * P, h->st);
    }
    for (int32_t u = 0; dd && u < nl; ++u) {
        const unsigned long long* dt = dd + (size_t)u * ((size_t)nr + 1);
        if (digests) copy_out(digests + u, dt, sizeof(uint64_t), h->st);
        if (row_digests) copy_out(row_digests + (size_t)u * nr, dt + 1, sizeof(uint64_t) * nr, h->st);
    }
    SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
    finish_timing(h, P);
    if (!dev) {
        slg::dfree(dI, h->st);
        slg::dfree(dJ, h->st);
        slg::dfree(dO, h->st);
    }
    slg::dfree(dd, h->st);
    API_END
}

slg_status slg_ensemble_stream_window(slg_graph* h, const int32_t* s_list, int32_t k, int32_t r0,
                                      int32_t* I, int32_t* J, int32_t* O, int64_t cap,
                                      int32_t* r1, int64_t* pairs) {
    if (!h || !r1 || !pairs) return fail(SLG_EINVAL, "NULL argument");
    if (r0 < 0 || r0 > h->g.m) return fail(SLG_EINVAL, "bad row range");
    if (cap < 1) return fail(SLG_EINVAL, "cap must be >= 1");
    if (!I || !J || !O) return fail(SLG_EINVAL, "NULL output array");
    API_BEGIN
    check_s_list(h, s_list, k);
    if (!slg::is_device_ptr(I) || !slg::is_device_ptr(J) || !slg::is_device_ptr(O))
        throw Error{SLG_EINVAL, "one-walk windows write device arrays only"};
    slg::stream_window(h, s_list, k, r0, I, J, O, cap, r1, pairs);
    API_END
}

slg_status slg_stream_window(slg_graph* h, int32_t s, int32_t r0, int32_t* I, int32_t* J,
                             int32_t* O, int64_t cap, int32_t* r1, int64_t* pairs) {
    return slg_ensemble_stream_window(h, &s, 1, r0, I, J, O, cap, r1, pairs);
}

slg_status slg_set_timing(slg_graph* h, int32_t enable) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    h->timer.on = enable != 0;
    h->mtimer.on = enable != 0;
    return SLG_OK;
}

slg_status slg_kernel_stats(slg_graph* h, int32_t reset, float* ms, int64_t* launches) {
    static_assert(slg::NMODES == SLG_NMODES, "handler count");
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    for (int pass = 0; pass < 2; ++pass)
        for (int k = 0; k < slg::NMODES; ++k) {
            if (ms) ms[pass * slg::NMODES + k] = h->mtimer.ms[pass][k];
            if (launches) launches[pass * slg::NMODES + k] = h->mtimer.launches[pass][k];
            if (reset) {
                h->mtimer.ms[pass][k] = 0;
                h->mtimer.launches[pass][k] = 0;
            }
        }
    return SLG_OK;
}

slg_status slg_ensemble_fill_stats(slg_graph* h, int32_t reset, int64_t* out) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    static_assert(slg::ENS_MAX == SLG_ENSEMBLE_MAX, "ensemble size");
    for (int t = 0; t < slg::ENS_MAX; ++t)
        for (int c = 0; c < 6; ++c) {
            if (out) out[t * 6 + c] = h->ens_made[t][c];
            if (reset) h->ens_made[t][c] = 0;
        }
    return SLG_OK;
}

slg_status slg_mode_stats(slg_graph* h, int32_t s, int64_t* out) {
    if (!h || !out) return fail(SLG_EINVAL, "NULL argument");
    API_BEGIN
    ensure_counted(h, s);
    static_assert(slg::MS_COLS == SLG_MODE_STATS_COLS, "mode statistics columns");
    int64_t st[slg::NMODES][slg::MS_COLS];
    slg::plan_mode_stats(h->g, h->plan, st, h->st);
    for (int k = 0; k < slg::NMODES; ++k)
        for (int c = 0; c < slg::MS_COLS; ++c) out[k * slg::MS_COLS + c] = st[k][c];
    API_END
}

slg_status slg_ensemble_mode_stats(slg_graph* h, const int32_t* s_list, int32_t k, int32_t which,
                                   int64_t* out) {
    if (!h || !out) return fail(SLG_EINVAL, "NULL argument");
    if (which < 0 || which >= k) return fail(SLG_EINVAL, "bad list selector");
    API_BEGIN
    ensure_ensemble(h, s_list, k);
    const slg::Plan& p = h->plan;
    int64_t st[slg::NMODES][slg::MS_COLS];
    slg::plan_mode_stats(h->g, p, st, h->st, p.ens.rowoff + (int64_t)which * ((int64_t)h->g.m + 1),
                         p.ens.ioff + (int64_t)which * (p.nitems + 1));
    for (int q = 0; q < slg::NMODES; ++q)
        for (int c = 0; c < slg::MS_COLS; ++c) out[q * slg::MS_COLS + c] = st[q][c];
    API_END
}

int64_t slg_kernel_launches(void) { return (int64_t)slg::g_launches.load(); }

slg_status slg_last_timing(slg_graph* h, float* ms5) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    if (ms5) memcpy(ms5, h->ms, sizeof(h->ms));
    return SLG_OK;
}

slg_status slg_set_bins(slg_graph* h, int32_t warp_max_wedges, int32_t block_item_wedges,
                        int32_t dense_min_density, int32_t dense_item_tiles,
                        int32_t wdense_max_ranges, int32_t sparse_min_per_tile,
                        int32_t sparse_item_wedges, int32_t wsparse_max_size) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    if (warp_max_wedges < 0 || warp_max_wedges > slg::WARP_TABLE / 2 || block_item_wedges < 1 ||
        dense_item_tiles < 1 || dense_item_tiles > 4096 || wdense_max_ranges < 0 ||
        wdense_max_ranges > slg::WD_MAXR || sparse_item_wedges < 1 || wsparse_max_size < 0 ||
        wsparse_max_size > slg::WS_MAXE)
        return fail(SLG_EINVAL, "bin parameter out of range");
    API_BEGIN
    h->bp.warp_max_wedges = warp_max_wedges;
    h->bp.block_item_wedges = block_item_wedges;
    h->bp.dense_min_density = dense_min_density;
    h->bp.dense_item_tiles = dense_item_tiles;
    h->bp.wdense_max_ranges = wdense_max_ranges;
    h->bp.sparse_min_per_tile = sparse_min_per_tile;
    h->bp.sparse_item_wedges = sparse_item_wedges;
    h->bp.wsparse_max_size = wsparse_max_size;
    h->plan.release(h->st);
    API_END
}

slg_status slg_set_hub_pairs(slg_graph* h, int32_t max_hubs, int64_t min_sparse_wedges) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    if (max_hubs < 0 || max_hubs > slg::HP_MAXK || min_sparse_wedges < 0)
        return fail(SLG_EINVAL, "max_hubs must be in [0, 4096], min_sparse_wedges >= 0");
    API_BEGIN
    h->plan.release(h->st);
    h->hp.release(h->st);
    h->hp.tried = false;
    h->hp_max_hubs = max_hubs;
    h->hp_min_wedges = min_sparse_wedges;
    API_END
}

slg_status slg_set_ensemble_filter(slg_graph* h, int32_t mode) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    if (mode < -1 || mode > 1) return fail(SLG_EINVAL, "mode must be -1 (automatic), 0 or 1");
    h->ens_filter = mode;
    slg::g_last_error.clear();
    return SLG_OK;
}

slg_status slg_set_staging(slg_graph* h, int64_t max_bytes) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    if (max_bytes < -1) return fail(SLG_EINVAL, "max_bytes must be -1 (automatic), 0 (off) or > 0");
    API_BEGIN
    h->plan.release(h->st);
    h->stage_max_bytes = max_bytes;
    API_END
}

slg_status slg_staging_stats(slg_graph* h, int64_t* out4) {
    if (!h || !out4) return fail(SLG_EINVAL, "graph and out4 must not be NULL");
    API_BEGIN
    const slg::Plan& p = h->plan;
    const bool on = (p.counted || p.ens.counted) && p.stage_at;
    out4[0] = on ? p.stage_cap : 0;
    out4[1] = on ? p.stage_chunk : 0;
    out4[2] = on ? slg::plan_staged_items(p, h->st) : 0;
    out4[3] = p.built ? p.nitems : 0;
    API_END
}

slg_status slg_autotune(slg_graph* h, int32_t s, int32_t max_trials, int32_t* bins_out,
                        float* ms_out) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    if (max_trials < 1) return fail(SLG_EINVAL, "max_trials must be >= 1");
    API_BEGIN
    check_s(h, s);
    slg::autotune(h, s, max_trials, ms_out);
    if (bins_out) {
        const slg::BinParams& b = h->bp;
        const int32_t v[8] = {b.warp_max_wedges,     b.block_item_wedges, b.dense_min_density,
                              b.dense_item_tiles,    b.wdense_max_ranges, b.sparse_min_per_tile,
                              b.sparse_item_wedges,  b.wsparse_max_size};
        for (int c = 0; c < 8; ++c) bins_out[c] = v[c];
    }
    API_END
}

slg_status slg_batch_load(slg_graph* const* gs, const int32_t* s, int32_t k, void* stream,
                          slg_graph** out) {
    if (!out) return fail(SLG_EINVAL, "out is NULL");
    *out = nullptr;
    if (k < 1 || !gs || !s) return fail(SLG_EINVAL, "need k >= 1 graphs and their s");
    int64_t M = 0, N = 0, NNZ = 0;
    int32_t min_size = INT32_MAX, max_size = 0;
    std::vector<slg::BatchPart> parts((size_t)k);
    for (int32_t b = 0; b < k; ++b) {
        const slg_graph* m = gs[b];
        if (!m) return fail(SLG_EINVAL, "NULL member graph");
        if (m->g.srow) return fail(SLG_EINVAL, "a batch cannot contain a batch");
        if (s[b] < 1) return fail(SLG_EINVAL, "every member's s must be >= 1");
        slg::BatchPart& P = parts[(size_t)b];
        P.off = m->g.off;
        P.idx = m->g.idx;
        P.size = m->g.size;
        P.rowid = m->g.rowid;
        P.offT = m->g.offT;
        P.idxT = m->g.idxT;
        P.tpos = m->g.tpos;
        P.hubidx = m->g.hubidx;
        P.hubmask = m->g.hubmask;
        P.m = m->g.m;
        P.n = m->g.n;
        P.nnz = m->g.nnz;
        P.row_base = (int32_t)M;
        P.vert_base = (int32_t)N;
        P.nnz_base = NNZ;
        P.s = s[b];
        M += m->g.m;
        N += m->g.n;
        NNZ += m->g.nnz;
        if (M >= INT32_MAX || N >= INT32_MAX || NNZ >= INT32_MAX)
            return fail(SLG_EINVAL, "the batch exceeds 2^31 rows, vertices or incidences");
        if (m->g.min_size > 0) min_size = std::min(min_size, m->g.min_size);
        max_size = std::max(max_size, m->g.max_size);
    }
    slg_graph* h = new slg_graph();
    h->st = (cudaStream_t)stream;
    // a batch's many small graphs gain nothing from staging (measured on the
    // 4,096-graph batch) and its pool would stay with the batch's plan
    h->stage_max_bytes = 0;
    try {
        SLG_CUDA_TRY(cudaGetDevice(&h->device));
        slg::GraphDev& g = h->g;
        g.m = (int32_t)M;
        g.n = (int32_t)N;
        g.nnz = NNZ;
        g.min_size = min_size == INT32_MAX ? 0 : min_size;
        g.max_size = max_size;
        g.off = slg::dalloc<int32_t>((size_t)M + 1, h->st);
        g.idx = slg::dalloc<int32_t>((size_t)NNZ + 4, h->st);
        g.size = slg::dalloc<int32_t>((size_t)M, h->st);
        g.rowid = slg::dalloc<int32_t>((size_t)NNZ + 4, h->st);
        g.offT = slg::dalloc<int32_t>((size_t)N + 1, h->st);
        g.idxT = slg::dalloc<int32_t>((size_t)NNZ + 4, h->st);
        g.tpos = slg::dalloc<int32_t>((size_t)NNZ + 4, h->st);
        g.srow = slg::dalloc<int32_t>((size_t)M, h->st);
        g.rbase = slg::dalloc<int32_t>((size_t)M, h->st);
        SLG_CUDA_TRY(cudaMemsetAsync(g.idxT + NNZ, 0, sizeof(int32_t) * 4, h->st));
        g.hubidx = slg::dalloc<int32_t>((size_t)N + 1, h->st);
        g.hubmask = slg::dalloc<uint32_t>((size_t)M + 64, h->st);
        SLG_CUDA_TRY(cudaMemsetAsync(g.hubmask, 0, sizeof(uint32_t) * ((size_t)M + 64), h->st));
        slg::BatchPart* parts_dev = slg::dalloc<slg::BatchPart>((size_t)k, h->st);
        SLG_CUDA_TRY(cudaMemcpyAsync(parts_dev, parts.data(), sizeof(slg::BatchPart) * k,
                                     cudaMemcpyHostToDevice, h->st));
        slg::launch_concat(parts_dev, k, (int32_t)M, (int32_t)N, NNZ, g, h->st);
        g.nhubs = slg::MAX_HUBS;  // per member
        SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
        slg::dfree(parts_dev, h->st);
        h->batch_row_base.resize((size_t)k + 1);
        for (int32_t b = 0; b < k; ++b) h->batch_row_base[(size_t)b] = parts[(size_t)b].row_base;
        h->batch_row_base[(size_t)k] = (int32_t)M;
        h->timer.init();
        slg::mtimer_init(h->mtimer);
    } catch (const Error& e) {
        free_graph_dev(h->g, h->st);
        cudaStreamSynchronize(h->st);
        delete h;
        return fail(e.code, e.msg);
    }
    *out = h;
    slg::g_last_error.clear();
    return SLG_OK;
}

slg_status slg_batch_info(const slg_graph* h, int32_t* k, int32_t* row_base) {
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    if (h->batch_row_base.empty()) return fail(SLG_EINVAL, "not a batch");
    const int32_t kk = (int32_t)h->batch_row_base.size() - 1;
    if (k) *k = kk;
    if (row_base) memcpy(row_base, h->batch_row_base.data(), sizeof(int32_t) * ((size_t)kk + 1));
    return SLG_OK;
}

slg_status slg_batch_pair_offsets(slg_graph* h, int64_t* pair_base) {
    if (!h || !pair_base) return fail(SLG_EINVAL, "NULL argument");
    if (h->batch_row_base.empty()) return fail(SLG_EINVAL, "not a batch");
    API_BEGIN
    ensure_counted(h, 0);
    const int32_t k = (int32_t)h->batch_row_base.size() - 1;
    int32_t* rb = slg::dalloc<int32_t>((size_t)k + 1, h->st);
    int64_t* po = slg::dalloc<int64_t>((size_t)k + 1, h->st);
    SLG_CUDA_TRY(cudaMemcpyAsync(rb, h->batch_row_base.data(), sizeof(int32_t) * ((size_t)k + 1),
                                 cudaMemcpyHostToDevice, h->st));
    slg::launch_gather_offsets(h->plan.rowoff, rb, k, po, h->st);
    copy_out(pair_base, po, sizeof(int64_t) * ((size_t)k + 1), h->st);
    SLG_CUDA_TRY(cudaStreamSynchronize(h->st));
    slg::dfree(rb, h->st);
    slg::dfree(po, h->st);
    API_END
}

void slg_result_free(slg_result* r) {
    if (!r) return;
    free(r->I);
    free(r->J);
    free(r->O);
    r->I = r->J = r->O = nullptr;
}

slg_status slg_batch(slg_graph* const* gs, const int32_t* s, int32_t k, slg_result* res) {
    if (!res) return fail(SLG_EINVAL, "results is NULL");
    if (k < 1 || !gs || !s) return fail(SLG_EINVAL, "need k >= 1 graphs and their s");
    for (int32_t b = 0; b < k; ++b) {
        res[b].status = SLG_OK;
        res[b].pairs = res[b].wedges = 0;
        res[b].digest = 0;
        res[b].I = res[b].J = res[b].O = nullptr;
    }
    auto fail_all = [&](slg_status code) {
        for (int32_t b = 0; b < k; ++b) {
            slg_result_free(&res[b]);
            res[b].status = code;
        }
        return code;
    };
    if (!gs[0]) return fail_all(fail(SLG_EINVAL, "NULL member graph"));
    slg_graph* h = nullptr;
    slg_status rc = slg_batch_load(gs, s, k, gs[0]->st, &h);
    if (rc != SLG_OK) return fail_all(rc);
    cudaStream_t st = h->st;
    int32_t* rb_dev = nullptr;
    long long* wsum = nullptr;
    unsigned long long *dsum = nullptr, *rowdig = nullptr;
    int32_t *dI = nullptr, *dJ = nullptr, *dO = nullptr;
    try {
        ensure_counted(h, 0);
        const int32_t M = h->g.m;
        const std::vector<int32_t>& rb = h->batch_row_base;
        std::vector<int64_t> pbase((size_t)k + 1);
        rc = slg_batch_pair_offsets(h, pbase.data());
        if (rc != SLG_OK) throw Error{rc, slg::g_last_error};
        // every row's digest, then per-member sums of W and digests
        rowdig = slg::dalloc<unsigned long long>((size_t)M + 1, st);
        SLG_CUDA_TRY(cudaMemsetAsync(rowdig, 0, sizeof(unsigned long long) * ((size_t)M + 1), st));
        const int64_t total = h->plan.pairs;
        const int64_t maxrow = slg::plan_max_row(h->g, h->plan.rowoff, st);
        const int64_t cap = std::max<int64_t>(maxrow, std::min<int64_t>(total, (int64_t)1 << 27));
        if (total > 0) {
            dI = slg::dalloc<int32_t>((size_t)cap, st);
            dJ = slg::dalloc<int32_t>((size_t)cap, st);
            dO = slg::dalloc<int32_t>((size_t)cap, st);
        }
        for (int32_t b = 0; b < k; ++b) {
            const int64_t n = pbase[(size_t)b + 1] - pbase[(size_t)b];
            if (!res[b].want_list || n == 0) continue;
            res[b].I = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
            res[b].J = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
            res[b].O = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
            if (!res[b].I || !res[b].J || !res[b].O)
                throw Error{SLG_ENOMEM, "no host memory for a member's list"};
        }
        std::vector<int32_t> splits((size_t)M + 2, 0);
        int32_t nw = 0;
        if (M > 0) {
            rc = slg_plan_windows(h, 0, std::max<int64_t>(cap, 1), splits.data(), M + 1, &nw);
            if (rc != SLG_OK) throw Error{rc, slg::g_last_error};
        }
        for (int32_t w = 0; w < nw; ++w) {
            const int32_t r0 = splits[(size_t)w], r1 = splits[(size_t)w + 1];
            int64_t Pw = 0;
            rc = slg_build_window(h, 0, r0, r1, dI, dJ, dO, cap, &Pw, nullptr,
                                  reinterpret_cast<uint64_t*>(rowdig) + r0);
            if (rc != SLG_OK) throw Error{rc, slg::g_last_error};
            if (Pw == 0) continue;
            // the window's list is the slice [wbase, wbase + Pw) of the batch's
            int64_t wbase = 0;
            SLG_CUDA_TRY(cudaMemcpyAsync(&wbase, h->plan.rowoff + r0, sizeof(int64_t),
                                         cudaMemcpyDeviceToHost, st));
            SLG_CUDA_TRY(cudaStreamSynchronize(st));
            const int32_t b0 = (int32_t)(std::upper_bound(rb.begin(), rb.end(), r0) - rb.begin()) - 1;
            for (int32_t b = std::max(b0, 0); b < k && rb[(size_t)b] < r1; ++b) {
                if (!res[b].I) continue;
                const int64_t a = std::max(pbase[(size_t)b], wbase);
                const int64_t z = std::min(pbase[(size_t)b + 1], wbase + Pw);
                if (z <= a) continue;
                const size_t bytes = sizeof(int32_t) * (size_t)(z - a);
                const int64_t to = a - pbase[(size_t)b], from = a - wbase;
                copy_out(res[b].I + to, dI + from, bytes, st);
                copy_out(res[b].J + to, dJ + from, bytes, st);
                copy_out(res[b].O + to, dO + from, bytes, st);
            }
            SLG_CUDA_TRY(cudaStreamSynchronize(st));
        }
        rb_dev = slg::dalloc<int32_t>((size_t)k + 1, st);
        wsum = slg::dalloc<long long>((size_t)k, st);
        dsum = slg::dalloc<unsigned long long>((size_t)k, st);
        SLG_CUDA_TRY(cudaMemcpyAsync(rb_dev, rb.data(), sizeof(int32_t) * ((size_t)k + 1),
                                     cudaMemcpyHostToDevice, st));
        slg::launch_member_sums(h->plan.W, rowdig, rb_dev, k, wsum, dsum, st);
        std::vector<long long> wh((size_t)k);
        std::vector<unsigned long long> dh((size_t)k);
        copy_out(wh.data(), wsum, sizeof(long long) * (size_t)k, st);
        copy_out(dh.data(), dsum, sizeof(unsigned long long) * (size_t)k, st);
        SLG_CUDA_TRY(cudaStreamSynchronize(st));
        for (int32_t b = 0; b < k; ++b) {
            res[b].pairs = pbase[(size_t)b + 1] - pbase[(size_t)b];
            res[b].wedges = (int64_t)wh[(size_t)b];
            res[b].digest = (uint64_t)dh[(size_t)b];
        }
    } catch (const Error& e) {
        rc = e.code;
        slg::set_error(e.code, e.msg);
    }
    slg::dfree(dI, st);
    slg::dfree(dJ, st);
    slg::dfree(dO, st);
    slg::dfree(rowdig, st);
    slg::dfree(rb_dev, st);
    slg::dfree(wsum, st);
    slg::dfree(dsum, st);
    const std::string msg = slg::g_last_error;
    slg_free(h);
    if (rc != SLG_OK) {
        slg::g_last_error = msg;
        return fail_all(rc);
    }
    slg::g_last_error.clear();
    return SLG_OK;
}

slg_status slg_dual(slg_graph* h, void* stream, slg_graph** out) {
    if (!out) return fail(SLG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!h) return fail(SLG_EINVAL, "graph is NULL");
    if (h->g.srow) return fail(SLG_EINVAL, "the dual of a batch is not defined");
    // the dual's incidence is this graph's transpose, already on the device
    return slg_load(h->g.offT, h->g.idxT, h->g.n, h->g.m, stream, out);
}

}  // extern "C"

