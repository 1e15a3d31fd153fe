// Negative-sampling LINE loss over a fixed set of samples (draw domain 3):
// terms[t] = -(log sigma(s+) + sum_j log sigma(-s-_j)), s = U[u].Ctx[y] in
// FP64 from the stored values.  The caller reduces terms[] with the
// fixed-order FP64 sum, so the loss is reproducible.
#include <math.h>

#include "line_internal.cuh"

namespace line {

namespace {

__device__ __forceinline__ double load_elem(const void* p, int dtype, int64_t idx) {
    return dtype == LINE_DTYPE_F32 ? (double)reinterpret_cast<const float*>(p)[idx]
                                   : (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[idx]);
}

// log sigma(s) = -(max(-s, 0) + log1p(exp(-|s|)))
__device__ __forceinline__ double log_sigmoid(double s) {
    const double a = s < 0.0 ? -s : 0.0;
    return -(a + log1p(exp(-fabs(s))));
}

// One warp per sample; lanes split the dimension, FP64 partial dots reduced
// in a fixed butterfly order.
__global__ void k_loss_terms(const void* __restrict__ U, const void* __restrict__ Ctx, int dtype, int dim, int K,
                             const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                             const uint2* __restrict__ edge_tab, int64_t n_arcs, const uint2* __restrict__ neg_tab,
                             int64_t n_nodes, uint64_t seed, int64_t m, double* __restrict__ terms) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < m; t += warps) {
        const uint4 w0 = draw_words(seed, 3u, (uint64_t)t, 0u);
        const uint32_t e = alias_pick(edge_tab, (uint64_t)n_arcs, w0);
        const int64_t u = src[e];
        double L = 0.0;
        for (int j = 0; j <= K; ++j) {
            int64_t y;
            if (j == 0) {
                y = dst[e];
            } else {
                y = alias_pick(neg_tab, (uint64_t)n_nodes, draw_words(seed, 3u, (uint64_t)t, (uint32_t)j));
            }
            double part = 0.0;
            for (int k = lane; k < dim; k += 32) part += load_elem(U, dtype, u * dim + k) * load_elem(Ctx, dtype, y * dim + k);
            for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
            L -= j == 0 ? log_sigmoid(part) : log_sigmoid(-part);
        }
        if (lane == 0) terms[t] = L;
    }
}

}  // namespace

cudaError_t eval_loss_terms(const void* U, const void* Ctx, int dtype, int dim, int K, const int32_t* src,
                            const int32_t* dst, const uint2* edge_tab, int64_t n_arcs, const uint2* neg_tab,
                            int64_t n_nodes, uint64_t seed, int64_t m, double* terms, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    int64_t blocks = (m + 7) / 8;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_loss_terms<<<(unsigned)blocks, 256, 0, s>>>(U, Ctx, dtype, dim, K, src, dst, edge_tab, n_arcs, neg_tab, n_nodes,
                                                  seed, m, terms);
    return cudaGetLastError();
}

}  // namespace line
