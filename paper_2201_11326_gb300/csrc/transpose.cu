// Load-time kernels: CSR validation and the dual incidence H^T.
//
// H^T (Section II-A: the dual hypergraph has the transposed incidence) is
// what the "ikj" loop order of Section III-B walks: for k in H^T.Adj[i], for j
// in H.Adj[k]. Here adj(v) must list hyperedges in increasing id so that the
// wedges (i, v, j) with j > i form a suffix of adj(v) (the i < j upper
// triangle of Section IV, Stage 1).
//
// The transpose is a stable counting sort of the incidences by vertex id
// (least-significant-digit radix, 8-bit digits): incidences arrive in
// increasing hyperedge order, and a stable sort by v keeps that order inside
// each adj(v). Besides offT/idxT it records tpos[e], the position of
// incidence e inside H^T, from which pruned positions are derived per s.
#include "slg_internal.cuh"

namespace slg {
namespace {

constexpr int VAL_THREADS = 256;

// flag bits
constexpr int32_t BAD_OFFSETS = 1;
constexpr int32_t BAD_ID = 2;
constexpr int32_t BAD_ORDER = 4;

__global__ void k_check_offsets(const int32_t* __restrict__ off, int32_t m, int64_t nnz,
                                int32_t* __restrict__ size, int32_t* __restrict__ flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int32_t a = off[i], b = off[i + 1];
        if (b < a || a < 0 || (int64_t)b > nnz) {
            atomicOr(flag, BAD_OFFSETS);
            size[i] = 0;
        } else {
            size[i] = b - a;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (off[0] != 0 || (int64_t)off[m] != nnz) atomicOr(flag, BAD_OFFSETS);
    }
}

// One warp per row writes rowid for the row's incidences. Offsets are
// clamped to [0, nnz] so that a malformed CSR (reported by k_check_offsets)
// cannot make this kernel write out of bounds.
__global__ void k_rowid(const int32_t* __restrict__ off, int32_t m, int64_t nnz,
                        int32_t* __restrict__ rowid) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < m; i += nwarps) {
        int64_t a = off[i], b = off[i + 1];
        a = a < 0 ? 0 : (a > nnz ? nnz : a);
        b = b < a ? a : (b > nnz ? nnz : b);
        for (int64_t e = a + lane; e < b; e += 32) rowid[e] = (int32_t)i;
    }
}

// Ids in [0, n) and strictly increasing inside each row.
__global__ void k_check_ids(const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                            const int32_t* __restrict__ rowid, int32_t n, int64_t nnz,
                            int32_t* __restrict__ flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const int32_t v = idx[e];
        if (v < 0 || v >= n) atomicOr(flag, BAD_ID);
        const int32_t i = rowid[e];
        if (e > off[i] && idx[e - 1] >= v) atomicOr(flag, BAD_ORDER);
    }
}

// ------------------------------------------------------------ degree count

// deg[v] += 1 per incidence; lanes holding the same v in a warp combine their
// increments first (hub vertices otherwise serialise on one address).
__global__ void k_degree(const int32_t* __restrict__ idx, int64_t nnz, int32_t* __restrict__ deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nnz; base += stride) {
        const int64_t e = base + threadIdx.x;
        const bool ok = e < nnz;
        const int32_t v = ok ? idx[e] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, v);
        const int leader = __ffs(peers) - 1;
        if (ok && lane == leader) atomicAdd(&deg[v], __popc(peers));
    }
}

// -------------------------------------------------------------- radix sort

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_IPT = 16;                       // items per thread
constexpr int RS_TILE = RS_THREADS * RS_IPT;     // 4096 items per CTA
constexpr int RS_SUB = RS_TILE / RS_WARPS;       // 512 items per warp
constexpr int RS_BINS = 256;

// Digit histogram of one tile, written digit-major: hist[d * ntiles + tile].
// keys == nullptr means the keys are idx (first pass).
__global__ void __launch_bounds__(RS_THREADS)
k_rs_hist(const int32_t* __restrict__ keys, int64_t nnz, int shift, int64_t ntiles,
          int32_t* __restrict__ hist) {
    __shared__ int32_t h[RS_BINS];
    for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_IPT; ++r) {
        const int64_t k = base + r * RS_THREADS + threadIdx.x;
        if (k < nnz) atomicAdd(&h[(keys[k] >> shift) & (RS_BINS - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS)
        hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// Stable scatter of one tile. Warp w owns items [w*RS_SUB, (w+1)*RS_SUB) of
// the tile and walks them in order 32 at a time, so ranks grow with position.
// vals_in == nullptr means the values are the positions themselves (first
// pass: value = incidence index).
__global__ void __launch_bounds__(RS_THREADS)
k_rs_scatter(const int32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
             int64_t nnz, int shift, int64_t ntiles, const int32_t* __restrict__ hist_off,
             int32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out) {
    __shared__ int32_t wh[RS_WARPS][RS_BINS];
    __shared__ int32_t tile_off[RS_BINS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < RS_WARPS * RS_BINS; t += RS_THREADS) (&wh[0][0])[t] = 0;
    for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS)
        tile_off[d] = hist_off[(int64_t)d * ntiles + blockIdx.x];
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * RS_SUB;
    const unsigned lt = (1u << lane) - 1u;
    int32_t key[RS_IPT], val[RS_IPT], rank[RS_IPT];
#pragma unroll
    for (int r = 0; r < RS_IPT; ++r) {
        const int64_t k = base + r * 32 + lane;
        const bool ok = k < nnz;
        key[r] = ok ? keys_in[k] : 0;
        val[r] = ok ? (vals_in ? vals_in[k] : (int32_t)k) : 0;
        const int d = ok ? ((key[r] >> shift) & (RS_BINS - 1)) : RS_BINS + lane;  // unique sentinel
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        int32_t before = 0;
        if (ok) before = wh[warp][d];
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) wh[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    // exclusive prefix over warps, per digit
    for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) {
        int32_t run = 0;
        for (int w = 0; w < RS_WARPS; ++w) {
            const int32_t c = wh[w][d];
            wh[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_IPT; ++r) {
        const int64_t k = base + r * 32 + lane;
        if (k < nnz) {
            const int d = (key[r] >> shift) & (RS_BINS - 1);
            const int64_t pos = (int64_t)tile_off[d] + wh[warp][d] + rank[r];
            keys_out[pos] = key[r];
            vals_out[pos] = val[r];
        }
    }
}

// idxT[k] = row of the incidence at sorted position k; tpos[e] = k.
__global__ void k_finish_transpose(const int32_t* __restrict__ sorted_e,
                                   const int32_t* __restrict__ rowid, int64_t nnz,
                                   int32_t* __restrict__ idxT, int32_t* __restrict__ tpos) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride) {
        const int32_t e = sorted_e[k];
        idxT[k] = rowid[e];
        tpos[e] = (int32_t)k;
    }
}

// ------------------------------------------------------------------ hubs
//
// The highest-degree vertices ("hubs", at most MAX_HUBS) are summarised by a
// 32-bit mask per hyperedge, so that the dense handler gets their share of an
// overlap as one popcount. Which vertices are hubs never changes a result;
// the pick below is deterministic (degree descending, then id).

constexpr int HUB_CAND = 4096;

__global__ void k_deg_buckets(const int32_t* __restrict__ offT, int32_t n,
                              int32_t* __restrict__ hist) {
    __shared__ int32_t h[32];
    if (threadIdx.x < 32) h[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = offT[v + 1] - offT[v];
        if (d >= 2) atomicAdd(&h[31 - __clz(d)], 1);
    }
    __syncthreads();
    if (threadIdx.x < 32 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_hub_candidates(const int32_t* __restrict__ offT, int32_t n, int32_t dmin,
                                 unsigned long long* __restrict__ cand,
                                 int32_t* __restrict__ ncand) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = offT[v + 1] - offT[v];
        if (d >= dmin && d >= 2) {
            const int32_t slot = atomicAdd(ncand, 1);
            if (slot < HUB_CAND)
                cand[slot] = ((unsigned long long)(uint32_t)(INT32_MAX - d) << 32) | (uint32_t)v;
        }
    }
}

// One CTA: sort the candidates by (degree desc, id asc), number the first
// MAX_HUBS of them.
__global__ void __launch_bounds__(1024)
k_hub_pick(const unsigned long long* __restrict__ cand, const int32_t* __restrict__ ncand,
           int32_t* __restrict__ hubidx, int32_t* __restrict__ nhubs) {
    __shared__ unsigned long long buf[HUB_CAND];
    const int32_t c = min(*ncand, HUB_CAND);
    int32_t P = 1;
    while (P < c) P <<= 1;
    for (int32_t t = threadIdx.x; t < P; t += blockDim.x) buf[t] = t < c ? cand[t] : ~0ull;
    __syncthreads();
    for (int32_t k = 2; k <= P; k <<= 1) {
        for (int32_t jj = k >> 1; jj > 0; jj >>= 1) {
            for (int32_t t = threadIdx.x; t < P; t += blockDim.x) {
                const int32_t u = t ^ jj;
                if (u > t) {
                    const unsigned long long x = buf[t], y = buf[u];
                    if ((x > y) == ((t & k) == 0)) {
                        buf[t] = y;
                        buf[u] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    const int32_t h = min(c, MAX_HUBS);
    if (threadIdx.x < h) hubidx[(int32_t)(buf[threadIdx.x] & 0xffffffffu)] = threadIdx.x;
    if (threadIdx.x == 0) *nhubs = h;
}

__global__ void k_hub_masks(const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                            const int32_t* __restrict__ hubidx, int32_t m,
                            uint32_t* __restrict__ hubmask) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t mask = 0;
        for (int32_t e = off[i]; e < off[i + 1]; ++e) {
            const int32_t b = hubidx[idx[e]];
            if (b >= 0) mask |= 1u << b;
        }
        hubmask[i] = mask;
    }
}

int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 64) g = 152 * 64;
    return (int)g;
}

}  // namespace

void launch_validate(const int32_t* off, const int32_t* idx, int32_t m, int32_t n, int64_t nnz,
                     int32_t* rowid, int32_t* size, int32_t* flag, cudaStream_t st) {
    SLG_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int32_t), st));
    k_check_offsets<<<grid_for(m, VAL_THREADS), VAL_THREADS, 0, st>>>(off, m, nnz, size, flag);
    SLG_LAUNCH_CHECK();
    if (m > 0) {
        k_rowid<<<grid_for((int64_t)m * 32, VAL_THREADS), VAL_THREADS, 0, st>>>(off, m, nnz, rowid);
        SLG_LAUNCH_CHECK();
    }
    if (nnz > 0) {
        k_check_ids<<<grid_for(nnz, VAL_THREADS), VAL_THREADS, 0, st>>>(off, idx, rowid, n, nnz,
                                                                       flag);
        SLG_LAUNCH_CHECK();
    }
}

void build_transpose(const int32_t* idx, const int32_t* rowid, int32_t n, int64_t nnz,
                     int32_t* offT, int32_t* idxT, int32_t* tpos, cudaStream_t st) {
    // offT: degree histogram + exclusive scan
    int32_t* deg = nullptr;
    SLG_CUDA_TRY(cudaMallocAsync((void**)&deg, sizeof(int32_t) * ((size_t)n + 1), st));
    SLG_CUDA_TRY(cudaMemsetAsync(deg, 0, sizeof(int32_t) * ((size_t)n + 1), st));
    if (nnz > 0) {
        k_degree<<<grid_for(nnz, 256), 256, 0, st>>>(idx, nnz, deg);
        SLG_LAUNCH_CHECK();
    }
    scan_i32_to_i32(deg, offT, n, st);
    SLG_CUDA_TRY(cudaFreeAsync(deg, st));
    if (nnz == 0) return;

    // stable LSD radix sort of incidence positions by vertex id
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < (int64_t)n) ++bits;
    const int passes = (bits + 7) / 8;
    const int64_t ntiles = (nnz + RS_TILE - 1) / RS_TILE;
    int32_t *k0, *v0, *k1, *v1, *hist;
    SLG_CUDA_TRY(cudaMallocAsync((void**)&k0, sizeof(int32_t) * nnz, st));
    SLG_CUDA_TRY(cudaMallocAsync((void**)&v0, sizeof(int32_t) * nnz, st));
    SLG_CUDA_TRY(cudaMallocAsync((void**)&k1, sizeof(int32_t) * nnz, st));
    SLG_CUDA_TRY(cudaMallocAsync((void**)&v1, sizeof(int32_t) * nnz, st));
    SLG_CUDA_TRY(cudaMallocAsync((void**)&hist, sizeof(int32_t) * (RS_BINS * ntiles + 1), st));
    const int32_t* kin = idx;
    const int32_t* vin = nullptr;
    int32_t *kout = k0, *vout = v0;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_rs_hist<<<(unsigned)ntiles, RS_THREADS, 0, st>>>(kin, nnz, shift, ntiles, hist);
        SLG_LAUNCH_CHECK();
        scan_i32_to_i32(hist, hist, RS_BINS * ntiles, st);
        k_rs_scatter<<<(unsigned)ntiles, RS_THREADS, 0, st>>>(kin, vin, nnz, shift, ntiles, hist,
                                                              kout, vout);
        SLG_LAUNCH_CHECK();
        kin = kout;
        vin = vout;
        kout = (kout == k0) ? k1 : k0;
        vout = (vout == v0) ? v1 : v0;
    }
    k_finish_transpose<<<grid_for(nnz, 256), 256, 0, st>>>(vin, rowid, nnz, idxT, tpos);
    SLG_LAUNCH_CHECK();
    SLG_CUDA_TRY(cudaFreeAsync(k0, st));
    SLG_CUDA_TRY(cudaFreeAsync(v0, st));
    SLG_CUDA_TRY(cudaFreeAsync(k1, st));
    SLG_CUDA_TRY(cudaFreeAsync(v1, st));
    SLG_CUDA_TRY(cudaFreeAsync(hist, st));
}

int32_t build_hubs(const int32_t* off, const int32_t* idx, const int32_t* offT, int32_t m,
                   int32_t n, int32_t* hubidx, uint32_t* hubmask, cudaStream_t st) {
    SLG_CUDA_TRY(cudaMemsetAsync(hubidx, 0xff, sizeof(int32_t) * ((size_t)n + 1), st));
    int32_t* work = nullptr;  // [0..31] degree buckets, [32] candidates, [33] hubs
    unsigned long long* cand = nullptr;
    SLG_CUDA_TRY(cudaMallocAsync((void**)&work, sizeof(int32_t) * 34, st));
    SLG_CUDA_TRY(cudaMallocAsync((void**)&cand, sizeof(unsigned long long) * HUB_CAND, st));
    SLG_CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(int32_t) * 34, st));
    int32_t nh = 0;
    if (n > 0) {
        k_deg_buckets<<<grid_for(n, 256), 256, 0, st>>>(offT, n, work);
        SLG_LAUNCH_CHECK();
        int32_t hist[32];
        SLG_CUDA_TRY(cudaMemcpyAsync(hist, work, sizeof(hist), cudaMemcpyDeviceToHost, st));
        SLG_CUDA_TRY(cudaStreamSynchronize(st));
        // smallest power-of-two degree bound keeping at most HUB_CAND candidates
        int b = 31;
        int64_t cum = hist[31];
        while (b > 1 && cum + hist[b - 1] <= HUB_CAND) {
            --b;
            cum += hist[b];
        }
        if (cum > 0) {
            const int32_t dmin = b >= 31 ? INT32_MAX : (int32_t)(1u << b);
            k_hub_candidates<<<grid_for(n, 256), 256, 0, st>>>(offT, n, dmin, cand, work + 32);
            SLG_LAUNCH_CHECK();
            k_hub_pick<<<1, 1024, 0, st>>>(cand, work + 32, hubidx, work + 33);
            SLG_LAUNCH_CHECK();
            SLG_CUDA_TRY(cudaMemcpyAsync(&nh, work + 33, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                         st));
        }
    }
    if (m > 0) {
        k_hub_masks<<<grid_for(m, 256), 256, 0, st>>>(off, idx, hubidx, m, hubmask);
        SLG_LAUNCH_CHECK();
    }
    SLG_CUDA_TRY(cudaStreamSynchronize(st));
    SLG_CUDA_TRY(cudaFreeAsync(work, st));
    SLG_CUDA_TRY(cudaFreeAsync(cand, st));
    return nh;
}

}  // namespace slg
