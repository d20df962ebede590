// Device helpers shared by the counting and fill kernels (internal).
#pragma once

#include "slg_internal.cuh"

namespace slg {

// error flags a kernel raises in its scratch word (reported as SLG_EINTERNAL)
constexpr int32_t ERR_BOUNDS = 1;  // a fill write fell outside the window
constexpr int32_t ERR_TABLE = 2;   // a table had no free slot
constexpr int32_t ERR_DIGEST = 4;  // a pair's row lay outside the window

__device__ __forceinline__ int32_t lower_bound_dev(const int32_t* __restrict__ a, int32_t lo,
                                                   int32_t hi, int32_t x) {
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ float warp_sum_f(float x) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    return x;
}

template <int NT>
__device__ __forceinline__ int32_t block_excl_scan(int32_t x, int32_t* total, int32_t* tmp) {
    // tmp: NT/32 + 1 ints of shared memory
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) tmp[w] = inc;
    __syncthreads();
    if (w == 0) {
        int32_t v = lane < NT / 32 ? tmp[lane] : 0;
        int32_t vi = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, vi, d);
            if (lane >= d) vi += y;
        }
        if (lane < NT / 32) tmp[lane] = vi - v;
        if (lane == NT / 32 - 1) tmp[NT / 32] = vi;
    }
    __syncthreads();
    const int32_t r = tmp[w] + inc - x;
    *total = tmp[NT / 32];
    __syncthreads();
    return r;
}

}  // namespace slg
