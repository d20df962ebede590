// Batches: many hypergraphs, each with its own s, as one disjoint union.
//
// Rows are the independent units of Algorithm 2 (Section III-C) and two
// hyperedges of different member graphs share no vertex, so the s-line graph
// of the union is the union of the members' s-line graphs, each member keeping
// its own threshold. The union is assembled on the device from the members'
// CSR and transposes (already built when they were loaded): row, vertex and
// incidence ids are shifted by per-member bases. Hub numbers stay per member:
// rows of different members never pair, so every member keeps its own (up to
// 32) hubs and masks. One plan, one counting pass, one scan and one fill per
// window then serve every member at once.
#include "plan.cuh"

namespace slg {
namespace {

__global__ void k_concat(const BatchPart* __restrict__ parts, int32_t M, int32_t N, int64_t NNZ,
                         int32_t k, GraphDev out) {
    const BatchPart P = parts[blockIdx.y];
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = t0; i < P.m; i += stride) {
        const int64_t r = P.row_base + i;
        out.off[r] = (int32_t)(P.nnz_base + P.off[i]);
        out.size[r] = P.size[i];
        out.srow[r] = P.s;
        out.rbase[r] = P.row_base;
        out.hubmask[r] = P.hubmask[i];
    }
    for (int64_t e = t0; e < P.nnz; e += stride) {
        const int64_t x = P.nnz_base + e;
        out.idx[x] = P.vert_base + P.idx[e];
        out.rowid[x] = P.row_base + P.rowid[e];
        out.idxT[x] = P.row_base + P.idxT[e];
        out.tpos[x] = (int32_t)(P.nnz_base + P.tpos[e]);
    }
    for (int64_t v = t0; v < P.n; v += stride) {
        out.offT[P.vert_base + v] = (int32_t)(P.nnz_base + P.offT[v]);
        out.hubidx[P.vert_base + v] = P.hubidx[v];
    }
    if (blockIdx.y == k - 1 && t0 == 0) {
        out.off[M] = (int32_t)NNZ;
        out.offT[N] = (int32_t)NNZ;
    }
}

__global__ void k_gather_offsets(const int64_t* __restrict__ rowoff,
                                 const int32_t* __restrict__ row_base, int32_t k,
                                 int64_t* __restrict__ out) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= k;
         b += (int64_t)gridDim.x * blockDim.x)
        out[b] = rowoff[row_base[b]];
}

// One CTA per member b: the sums of W[r] and dig[r] (mod 2^64) over its rows
// row_base[b] .. row_base[b+1]-1.
__global__ void k_member_sums(const int64_t* __restrict__ W,
                              const unsigned long long* __restrict__ dig,
                              const int32_t* __restrict__ row_base,
                              long long* __restrict__ wsum, unsigned long long* __restrict__ dsum) {
    constexpr int NT = 256;
    __shared__ long long sw[NT / 32];
    __shared__ unsigned long long sd[NT / 32];
    const int b = blockIdx.x;
    long long w = 0;
    unsigned long long d = 0;
    for (int64_t r = (int64_t)row_base[b] + threadIdx.x; r < row_base[b + 1]; r += NT) {
        w += W[r];
        if (dig) d += dig[r];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        w += __shfl_xor_sync(0xffffffffu, w, o);
        d += __shfl_xor_sync(0xffffffffu, d, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sw[threadIdx.x >> 5] = w;
        sd[threadIdx.x >> 5] = d;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tw = 0;
        unsigned long long td = 0;
        for (int x = 0; x < NT / 32; ++x) {
            tw += sw[x];
            td += sd[x];
        }
        wsum[b] = tw;
        dsum[b] = td;
    }
}

}  // namespace

void launch_member_sums(const int64_t* W, const unsigned long long* rowdig,
                        const int32_t* row_base_dev, int32_t k, long long* wsum_dev,
                        unsigned long long* dsum_dev, cudaStream_t st) {
    if (k <= 0) return;
    k_member_sums<<<(unsigned)k, 256, 0, st>>>(W, rowdig, row_base_dev, wsum_dev, dsum_dev);
    SLG_LAUNCH_CHECK();
}

void launch_concat(const BatchPart* parts_dev, int32_t k, int32_t M, int32_t N, int64_t NNZ,
                   const GraphDev& out, cudaStream_t st) {
    if (k <= 0) return;
    dim3 grid(32, (unsigned)k);
    k_concat<<<grid, 256, 0, st>>>(parts_dev, M, N, NNZ, k, out);
    SLG_LAUNCH_CHECK();
}

void launch_gather_offsets(const int64_t* rowoff, const int32_t* row_base_dev, int32_t k,
                           int64_t* out_dev, cudaStream_t st) {
    k_gather_offsets<<<(k + 256) / 256, 256, 0, st>>>(rowoff, row_base_dev, k, out_dev);
    SLG_LAUNCH_CHECK();
}

}  // namespace slg
