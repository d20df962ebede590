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

}  // namespace

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
