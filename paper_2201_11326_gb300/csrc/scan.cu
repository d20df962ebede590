// Device-wide exclusive prefix sums (reduce -> scan block sums -> scan tiles).
//
// Used to turn per-vertex degrees into H^T offsets, per-position keep flags
// into pruned-transpose positions, and per-item pair counts into output
// offsets (the count-then-fill scheme that replaces the per-thread output
// lists merged at the end of Algorithm 2, Section III-C).
#include <mutex>

#include "slg_internal.cuh"

namespace slg {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_IPT;

template <typename T>
__device__ T warp_inclusive_scan(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

// Exclusive scan of one value per thread across the CTA; returns the CTA total
// through *total.
template <typename T>
__device__ T block_exclusive_scan(T x, T* total) {
    __shared__ T warp_tot[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_inclusive_scan(x);
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < SCAN_THREADS / 32 ? warp_tot[lane] : T(0);
        T wi = warp_inclusive_scan(w);
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = wi - w;
        if (lane == SCAN_THREADS / 32 - 1) *total = wi;
    }
    __syncthreads();
    T r = warp_tot[warp] + inc - x;
    __syncthreads();
    return r;
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(SCAN_THREADS)
k_tile_reduce(const Tin* __restrict__ in, int64_t n, Tout* __restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    Tout acc = 0;
#pragma unroll
    for (int r = 0; r < SCAN_IPT; ++r) {
        const int64_t k = base + r * SCAN_THREADS + threadIdx.x;
        if (k < n) acc += (Tout)in[k];
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    __shared__ Tout wsum[SCAN_THREADS / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        Tout t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += wsum[w];
        sums[blockIdx.x] = t;
    }
}

// Scans tile blockIdx.x of `in` with the offset tile_off[blockIdx.x] (or 0
// when tile_off is null) into out; the last tile also writes out[n].
// In-place use (in == out, same type) is allowed: a CTA reads its whole tile
// before writing.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(SCAN_THREADS)
k_tile_scan(const Tin* in, int64_t n, const Tout* tile_off, Tout* out) {
    __shared__ Tout buf[SCAN_TILE];
    __shared__ Tout total;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int r = 0; r < SCAN_IPT; ++r) {
        const int t = r * SCAN_THREADS + threadIdx.x;
        const int64_t k = base + t;
        buf[t] = k < n ? (Tout)in[k] : Tout(0);
    }
    __syncthreads();
    Tout v[SCAN_IPT];
    Tout run = 0;
#pragma unroll
    for (int r = 0; r < SCAN_IPT; ++r) {
        v[r] = buf[threadIdx.x * SCAN_IPT + r];
        run += v[r];
    }
    const Tout off0 = (tile_off ? tile_off[blockIdx.x] : Tout(0));
    Tout ex = block_exclusive_scan<Tout>(run, &total) + off0;
#pragma unroll
    for (int r = 0; r < SCAN_IPT; ++r) {
        buf[threadIdx.x * SCAN_IPT + r] = ex;
        ex += v[r];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < SCAN_IPT; ++r) {
        const int t = r * SCAN_THREADS + threadIdx.x;
        const int64_t k = base + t;
        if (k < n) out[k] = buf[t];
    }
    if (threadIdx.x == 0 && base + SCAN_TILE >= n) out[n] = off0 + total;
}

template <typename Tin, typename Tout>
void scan_impl(const Tin* in, Tout* out, int64_t n, cudaStream_t st) {
    if (n <= 0) {
        SLG_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(Tout), st));
        return;
    }
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        k_tile_scan<Tin, Tout><<<1, SCAN_THREADS, 0, st>>>(in, n, nullptr, out);
        SLG_LAUNCH_CHECK();
        return;
    }
    Tout* sums = nullptr;
    SLG_CUDA_TRY(cudaMallocAsync((void**)&sums, sizeof(Tout) * (nb + 1), st));
    k_tile_reduce<Tin, Tout><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, sums);
    SLG_LAUNCH_CHECK();
    scan_impl<Tout, Tout>(sums, sums, nb, st);
    k_tile_scan<Tin, Tout><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, sums, out);
    SLG_LAUNCH_CHECK();
    SLG_CUDA_TRY(cudaFreeAsync(sums, st));
}

}  // namespace

void scan_i32_to_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st) {
    scan_impl<int32_t, int32_t>(in, out, n, st);
}
void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t st) {
    scan_impl<int32_t, int64_t>(in, out, n, st);
}
void scan_i64_to_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st) {
    scan_impl<int64_t, int64_t>(in, out, n, st);
}

}  // namespace slg

// ------------------------------------------------------------------------
// Scan of per-row counts that allocates nothing.
//
// The same tile kernels as above, but the tile sums live in a fixed device
// array compiled into the library instead of stream-ordered allocations.
// Capacity: 32768 level-1 tile sums of 2048 counts each, i.e. at most
// 67,108,864 counts per call; 264 KiB of device memory per GPU that loads the
// library, held until the process exits.

namespace {

constexpr int64_t NOALLOC_TILES = 32768;
constexpr int64_t NOALLOC_MAX_N = NOALLOC_TILES * slg::SCAN_TILE;
constexpr int64_t NOALLOC_TILES2 = (NOALLOC_TILES + slg::SCAN_TILE - 1) / slg::SCAN_TILE;
constexpr int64_t NOALLOC_ELEMS = (NOALLOC_TILES + 1) + (NOALLOC_TILES2 + 1);
constexpr int NOALLOC_MAX_DEVICES = 64;

std::mutex g_noalloc_mutex;
long long* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

}  // namespace

// Tile sums of every call, on every device (host code must not use this name
// as an address: it resolves it with cudaGetSymbolAddress below).
static __device__ __align__(256) long long g_noalloc_scan_sums[NOALLOC_ELEMS];

namespace {

// Device address of the array on the current device, looked up once per
// device (the first call on each device does it).
long long* noalloc_sums_on(int dev) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        throw slg::Error{SLG_EINVAL, "device ordinal beyond the no-allocation table"};
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scan_sums);
        if (e != cudaSuccess)
            throw slg::Error{SLG_ECUDA,
                             std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)};
        g_noalloc_addr[dev] = static_cast<long long*>(p);
    }
    return g_noalloc_addr[dev];
}

// Device memory of the current device (or managed memory): the kernels may
// not dereference another GPU's memory, which needs no peer mapping to exist.
bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" slg_status slg_scan_counts_noalloc(const int32_t* counts, int64_t* offsets, int64_t n,
                                              void* stream) {
    using slg::Error;
    try {
        if (n < 0 || n > NOALLOC_MAX_N)
            throw Error{SLG_EINVAL, "n must be in [0, 67108864] for the no-allocation scan"};
        if (!offsets || (n > 0 && !counts)) throw Error{SLG_EINVAL, "NULL argument"};
        if (!on_device(offsets) || (n > 0 && !on_device(counts)))
            throw Error{SLG_EINVAL, "counts and offsets must be memory of the current device"};
        int dev = 0;
        SLG_CUDA_TRY(cudaGetDevice(&dev));
        long long* sums1 = noalloc_sums_on(dev);
        long long* sums2 = sums1 + NOALLOC_TILES + 1;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        using slg::k_tile_reduce;
        using slg::k_tile_scan;
        constexpr int T = slg::SCAN_THREADS;
        if (n == 0) {
            SLG_CUDA_TRY(cudaMemsetAsync(offsets, 0, sizeof(int64_t), st));
        } else {
            const int64_t nb1 = (n + slg::SCAN_TILE - 1) / slg::SCAN_TILE;
            int64_t* out = reinterpret_cast<int64_t*>(offsets);
            int64_t* s1 = reinterpret_cast<int64_t*>(sums1);
            int64_t* s2 = reinterpret_cast<int64_t*>(sums2);
            if (nb1 == 1) {
                k_tile_scan<int32_t, int64_t><<<1, T, 0, st>>>(counts, n, nullptr, out);
                SLG_LAUNCH_CHECK();
            } else {
                k_tile_reduce<int32_t, int64_t><<<(unsigned)nb1, T, 0, st>>>(counts, n, s1);
                SLG_LAUNCH_CHECK();
                const int64_t nb2 = (nb1 + slg::SCAN_TILE - 1) / slg::SCAN_TILE;
                if (nb2 == 1) {
                    k_tile_scan<int64_t, int64_t><<<1, T, 0, st>>>(s1, nb1, nullptr, s1);
                    SLG_LAUNCH_CHECK();
                } else {
                    k_tile_reduce<int64_t, int64_t><<<(unsigned)nb2, T, 0, st>>>(s1, nb1, s2);
                    SLG_LAUNCH_CHECK();
                    k_tile_scan<int64_t, int64_t><<<1, T, 0, st>>>(s2, nb2, nullptr, s2);
                    SLG_LAUNCH_CHECK();
                    k_tile_scan<int64_t, int64_t><<<(unsigned)nb2, T, 0, st>>>(s1, nb1, s2, s1);
                    SLG_LAUNCH_CHECK();
                }
                k_tile_scan<int32_t, int64_t><<<(unsigned)nb1, T, 0, st>>>(counts, n, s1, out);
                SLG_LAUNCH_CHECK();
            }
        }
    } catch (const Error& e) {
        slg::set_error(e.code, e.msg);
        return e.code;
    }
    return SLG_OK;
}

