// Draw export, alias export, table initialisation and row conversion.
#include "line_internal.cuh"

namespace line {

namespace {

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 64) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

// One thread per (sample, call): call 0 draws the arc (Algorithm 3's
// weight-proportional pick), calls 1..K the negatives from q (Eq. 1).
__global__ void k_sample_records(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                 const uint2* __restrict__ edge_tab, int64_t n_arcs,
                                 const uint2* __restrict__ neg_tab, int64_t n_nodes, uint64_t seed,
                                 uint32_t domain, uint64_t t0, int64_t count, int K, int32_t* __restrict__ out) {
    const int64_t total = count * (int64_t)(K + 1);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = q / (K + 1);
        const int c = (int)(q - s * (K + 1));
        const uint4 w = draw_words(seed, domain, t0 + (uint64_t)s, (uint32_t)c);
        int32_t* rec = out + s * (K + 2);
        if (c == 0) {
            const uint32_t e = alias_pick(edge_tab, (uint64_t)n_arcs, w);
            rec[0] = __ldg(src + e);
            rec[1] = __ldg(dst + e);
        } else {
            rec[1 + c] = (int32_t)alias_pick(neg_tab, (uint64_t)n_nodes, w);
        }
    }
}

__global__ void k_export_alias(const uint2* __restrict__ tab, int64_t n, uint32_t* __restrict__ thr,
                               uint32_t* __restrict__ alias) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint2 e = tab[i];
        thr[i] = e.x;
        alias[i] = e.y;
    }
}

// U[i][k] = ((w >> 8) - 2^23) * 2^-24 / dim, w = word (k mod 4) of the draw at
// counter (i_lo, i_hi, k/4, 1): uniform on [-0.5/dim, 0.5/dim).
__global__ void k_init_uniform(void* __restrict__ U, int dtype, int64_t n, int dim, uint64_t seed) {
    const int64_t quads = n * (int64_t)(dim / 4);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < quads; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / (dim / 4);
        const int k4 = (int)(q - i * (dim / 4));
        const uint4 w = draw_words(seed, 1u, (uint64_t)i, (uint32_t)k4);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int32_t qv = (int32_t)(ws[j] >> 8) - (1 << 23);
            // exact in FP32: |qv| < 2^23, and 2^-24 and dim are powers of two
            v[j] = ((float)qv * (1.0f / 16777216.0f)) / (float)dim;
        }
        if (dtype == LINE_DTYPE_F32) {
            reinterpret_cast<float4*>(U)[q] = make_float4(v[0], v[1], v[2], v[3]);
        } else {
            __nv_bfloat16* p = reinterpret_cast<__nv_bfloat16*>(U) + q * 4;
#pragma unroll
            for (int j = 0; j < 4; ++j) p[j] = __float2bfloat16_rn(v[j]);
        }
    }
}

__device__ __forceinline__ float load_as_f32(const void* p, int dtype, int64_t idx) {
    return dtype == LINE_DTYPE_F32 ? reinterpret_cast<const float*>(p)[idx]
                                   : __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[idx]);
}

// dst[row(r)][k] = src[r][k] with dtype conversion (F32 -> BF16 rounds to
// nearest even).  rows == nullptr: row(r) = r.
__global__ void k_convert_rows(const void* __restrict__ src, int src_dtype, void* __restrict__ dst, int dst_dtype,
                               const int32_t* __restrict__ rows, int64_t n_rows, int dim, int64_t n_nodes,
                               uint32_t* status) {
    const int64_t total = n_rows * (int64_t)dim;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / dim;
        const int k = (int)(q - r * dim);
        int64_t row = r;
        if (rows) {
            row = rows[r];
            if (row < 0 || row >= n_nodes) {
                atomicOr(status, DEV_ERR_INDEX);
                continue;
            }
        }
        const float v = load_as_f32(src, src_dtype, q);
        const int64_t o = row * dim + k;
        if (dst_dtype == LINE_DTYPE_F32) reinterpret_cast<float*>(dst)[o] = v;
        else reinterpret_cast<__nv_bfloat16*>(dst)[o] = __float2bfloat16_rn(v);
    }
}

// Waits for a flag that nothing sets; the bounded wait gives up after
// `limit` polls and records DEV_ERR_TIMEOUT.
__global__ void k_debug_wait(uint32_t* flag, int64_t limit, uint32_t* status) {
    const uint32_t zero = 0;
    if (!wait_geq(flag, 1u, limit, &zero)) atomicOr(status, DEV_ERR_TIMEOUT);
}

}  // namespace

cudaError_t sample_records(const int32_t* src, const int32_t* dst, const uint2* edge_tab, int64_t n_arcs,
                           const uint2* neg_tab, int64_t n_nodes, uint64_t seed, uint32_t domain, uint64_t t0,
                           int64_t count, int K, int32_t* out, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    k_sample_records<<<grid_for(count * (K + 1), 256), 256, 0, s>>>(src, dst, edge_tab, n_arcs, neg_tab, n_nodes,
                                                                     seed, domain, t0, count, K, out);
    return cudaGetLastError();
}

cudaError_t export_alias(const uint2* tab, int64_t n, uint32_t* thr, uint32_t* alias, cudaStream_t s) {
    k_export_alias<<<grid_for(n, 256), 256, 0, s>>>(tab, n, thr, alias);
    return cudaGetLastError();
}

cudaError_t init_table(void* U, int dtype, int64_t n, int dim, uint64_t seed, cudaStream_t s) {
    k_init_uniform<<<grid_for(n * (dim / 4), 256), 256, 0, s>>>(U, dtype, n, dim, seed);
    return cudaGetLastError();
}

cudaError_t convert_rows(const void* src, int src_dtype, void* dst, int dst_dtype, const int32_t* rows,
                         int64_t n_rows, int dim, int64_t n_nodes, uint32_t* status, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    k_convert_rows<<<grid_for(n_rows * dim, 256), 256, 0, s>>>(src, src_dtype, dst, dst_dtype, rows, n_rows, dim,
                                                                n_nodes, status);
    return cudaGetLastError();
}

cudaError_t debug_wait(uint32_t* flag, int64_t limit, uint32_t* status, cudaStream_t s) {
    k_debug_wait<<<1, 32, 0, s>>>(flag, limit, status);
    return cudaGetLastError();
}

}  // namespace line
