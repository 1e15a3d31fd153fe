// Link-prediction evaluation (reporting): scores of node pairs and the exact
// Mann-Whitney AUC of positive against negative pairs: held-out edges
// against non-edges, the measure of embedding quality this library reports
// (the paper's own, node classification by Micro/Macro-F1 in §V-C, needs
// node labels).  Over the requested
// orders o, with z(x) = [U_o[x]]_o the concatenated rows:
//
//   dot:     score(u, v) = z(u).z(v) = sum_o U_o[u].U_o[v]
//   cosine:  score(u, v) = n(u).n(v) / (|n(u)| |n(v)|),  n(x) = [U_o[x] / |U_o[x]|]_o
//
// (cosine: an all-zero row contributes a zero block, a zero concatenated
// vector scores 0).  Scores are FP32: per order the dot and the two squared
// norms are FP32 FMA chains over a lane's dimensions, reduced by a butterfly
// (every lane ends with the same bits).  The AUC then
// counts, in integers, the (positive, negative) pairs with neg < pos and with
// neg == pos: the negatives' order-preserving 32-bit keys are radix sorted and
// every positive key is located by binary search.
#include "line_internal.cuh"

namespace line {

namespace {

__device__ __forceinline__ float load_f(const void* p, int dtype, int64_t idx) {
    return dtype == LINE_DTYPE_F32 ? reinterpret_cast<const float*>(p)[idx]
                                   : __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[idx]);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Monotone map float -> uint32 (after -0 -> +0): a < b  <=>  key(a) < key(b).
__device__ __forceinline__ uint32_t order_key(float f) {
    uint32_t b = __float_as_uint(f == 0.0f ? 0.0f : f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// One warp per pair.
__global__ void k_pair_scores(ScoreTables t, int score, const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                              int64_t n, int64_t n_nodes, float* __restrict__ scores, uint32_t* __restrict__ keys,
                              uint32_t* status) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const int64_t u = src[i], v = dst[i];
        if (u < 0 || u >= n_nodes || v < 0 || v >= n_nodes) {
            if (lane == 0) {
                atomicOr(status, DEV_ERR_INDEX);
                scores[i] = 0.0f;
                keys[i] = order_key(0.0f);
            }
            continue;
        }
        float zz = 0.0f, cu = 0.0f, cv = 0.0f, dd = 0.0f;
        for (int o = 0; o < t.n; ++o) {
            const void* U = t.U[o];
            const int dim = t.dim[o], dt = t.dtype[o];
            float dot = 0.0f, nu = 0.0f, nv = 0.0f;
            for (int k = lane; k < dim; k += 32) {
                const float a = load_f(U, dt, u * dim + k), b = load_f(U, dt, v * dim + k);
                dot = fmaf(a, b, dot);
                nu = fmaf(a, a, nu);
                nv = fmaf(b, b, nv);
            }
            dot = warp_sum(dot);
            nu = warp_sum(nu);
            nv = warp_sum(nv);
            dd += dot;
            if (nu > 0.0f && nv > 0.0f) zz += dot / (sqrtf(nu) * sqrtf(nv));
            if (nu > 0.0f) cu += 1.0f;
            if (nv > 0.0f) cv += 1.0f;
        }
        const float sc = score == LINE_SCORE_DOT ? dd : (cu > 0.0f && cv > 0.0f) ? zz / sqrtf(cu * cv) : 0.0f;
        if (lane == 0) {
            if (!(sc == sc)) atomicOr(status, DEV_ERR_VALUE);
            scores[i] = sc;
            keys[i] = order_key(sc);
        }
    }
}

// ---- LSD radix sort of 32-bit keys, 8 bits per pass.  Tiles of kTile keys,
// one block each; per-tile digit counts are scanned digit-major, and the
// scatter ranks keys stably (in index order) within each tile.
constexpr int kThreads = 256;
constexpr int kRounds = 16;
constexpr int kTile = kThreads * kRounds;

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ hist) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kRounds; ++r) {
        const int64_t i = base + r * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of hist[0..total) in place, one block of 1024 threads.
__global__ void k_scan_hist(uint32_t* hist, int64_t total) {
    __shared__ uint32_t part[1024];
    const int64_t per = (total + 1023) / 1024;
    const int64_t lo = threadIdx.x * per, hi = min(lo + per, total);
    uint32_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += hist[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const uint32_t o = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0u;
        __syncthreads();
        part[threadIdx.x] += o;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (int64_t i = lo; i < hi; ++i) {
        const uint32_t c = hist[i];
        hist[i] = run;
        run += c;
    }
}

__global__ void k_radix_scatter(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n, int shift,
                                const uint32_t* __restrict__ offs) {
    __shared__ uint32_t wcnt[kThreads / 32][256];
    __shared__ uint32_t run[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run[threadIdx.x] = offs[(size_t)threadIdx.x * gridDim.x + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kRounds; ++r) {
        for (int w = 0; w < kThreads / 32; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t i = base + r * kThreads + threadIdx.x;
        const bool valid = i < n;
        const uint32_t key = valid ? in[i] : 0u;
        const uint32_t d = valid ? (key >> shift) & 0xFFu : 0x100u + lane;  // invalid lanes match nobody
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && lane == 31 - __clz(peers)) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            // thread t owns digit t: warp offsets within the round, then the
            // digit's running position
            uint32_t s = run[threadIdx.x];
            for (int w = 0; w < kThreads / 32; ++w) {
                const uint32_t c = wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = s;
                s += c;
            }
            run[threadIdx.x] = s;
        }
        __syncthreads();
        if (valid) out[wcnt[warp][d] + rank] = key;
        __syncthreads();
    }
}

// counts[0] += #(neg < pos), counts[1] += #(neg == pos) over the positives.
__global__ void k_auc_count(const uint32_t* __restrict__ pos, int64_t n_pos, const uint32_t* __restrict__ neg,
                            int64_t n_neg, unsigned long long* counts) {
    unsigned long long less = 0, eq = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pos; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = pos[i];
        int64_t lo = 0, hi = n_neg;
        while (lo < hi) {  // first negative >= k
            const int64_t mid = (lo + hi) >> 1;
            if (neg[mid] < k) lo = mid + 1;
            else hi = mid;
        }
        int64_t lo2 = lo, hi2 = n_neg;
        while (lo2 < hi2) {  // first negative > k
            const int64_t mid = (lo2 + hi2) >> 1;
            if (neg[mid] <= k) lo2 = mid + 1;
            else hi2 = mid;
        }
        less += (unsigned long long)lo;
        eq += (unsigned long long)(lo2 - lo);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        less += __shfl_xor_sync(0xFFFFFFFFu, less, o);
        eq += __shfl_xor_sync(0xFFFFFFFFu, eq, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(counts, less);
        atomicAdd(counts + 1, eq);
    }
}

int64_t tiles(int64_t n) { return (n + kTile - 1) / kTile; }

}  // namespace

// tmp layout: the two counters (first 256 bytes), keys [n], sort buffer
// [n_neg], digit counts [256 * tiles].
size_t auc_tmp_bytes(int64_t n_pos, int64_t n_neg) {
    const int64_t n = n_pos + n_neg;
    return 256 + sizeof(uint32_t) * (size_t)(n + n_neg + 256 * tiles(n_neg));
}

cudaError_t eval_auc(const ScoreTables& t, int score, const int32_t* src, const int32_t* dst, int64_t n_pos, int64_t n_neg,
                     int64_t n_nodes, float* scores, void* tmp, uint32_t* status, cudaStream_t s) {
    const int64_t n = n_pos + n_neg;
    unsigned long long* counts_dev = reinterpret_cast<unsigned long long*>(tmp);
    uint32_t* keys = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(tmp) + 256);
    uint32_t* alt = keys + n;
    uint32_t* hist = alt + n_neg;
    cudaError_t e;
    if ((e = cudaMemsetAsync(counts_dev, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    {
        int64_t blocks = (n + 7) / 8;
        if (blocks > 152 * 32) blocks = 152 * 32;
        k_pair_scores<<<(unsigned)blocks, 256, 0, s>>>(t, score, src, dst, n, n_nodes, scores, keys, status);
    }
    // sort the negatives' keys (keys[n_pos ..]); four passes leave them in place
    uint32_t* a = keys + n_pos;
    uint32_t* b = alt;
    const int64_t nt = tiles(n_neg);
    for (int shift = 0; shift < 32; shift += 8) {
        k_radix_hist<<<(unsigned)nt, kThreads, 0, s>>>(a, n_neg, shift, hist);
        k_scan_hist<<<1, 1024, 0, s>>>(hist, 256 * nt);
        k_radix_scatter<<<(unsigned)nt, kThreads, 0, s>>>(a, b, n_neg, shift, hist);
        uint32_t* x = a;
        a = b;
        b = x;
    }
    {
        int64_t blocks = (n_pos + 255) / 256;
        if (blocks > 152 * 8) blocks = 152 * 8;
        k_auc_count<<<(unsigned)blocks, 256, 0, s>>>(keys, n_pos, a, n_neg, counts_dev);
    }
    return cudaGetLastError();
}

}  // namespace line
