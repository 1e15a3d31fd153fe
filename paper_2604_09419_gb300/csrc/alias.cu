// Alias tables on the GPU for the two discrete distributions of the method:
//   - the positive-pair pick over arcs, proportional to the arc weight
//     (Algorithm 3: the discrete distribution over E_p / ||E_p||), and
//   - the negative distribution q(v) = d(v)^0.75 / sum_x d(x)^0.75 with d the
//     weighted out-degree (Section IV-A, Eq. 1).
// FP64 is used only for the degree sums and the normalisation; the table is
// built from exact integer masses so that every bucket probability is a known
// rational and the construction is reproducible bit for bit.
//
// Pairing (the sweep rule, written as prefix sums so that it runs in
// parallel): let lights be the items with m < 2^32 (deficit Q - m), heavies
// those with m > 2^32 (excess m - Q), both in index order, DP/EP the
// inclusive prefix sums of deficits/excesses.  Light number j takes as alias
// the first heavy k with EP[k] >= DP[j-1]; heavy k (not the last) becomes a
// light bucket at the first light j with DP[j] > EP[k], with threshold
// Q - (DP[j] - EP[k]) and alias heavy k+1.  This is exactly the table of the
// sequential sweep in which the current heavy item tops up the lights in
// order and, when its own mass drops below Q, is topped up by the next heavy
// item (Huebschle-Schneider and Sanders, "Parallel Weighted Random
// Sampling", ESA 2019, describe the same parallel split).
#include <math.h>

#include "line_internal.cuh"
#include "scan.cuh"

namespace line {

namespace {

// Fixed-order FP64 sum of one block of 1024 values: halving strides.
__global__ void __launch_bounds__(kSumBlock / 2) k_tree_sum(const double* __restrict__ x, int64_t n,
                                                             double* __restrict__ out) {
    __shared__ double buf[kSumBlock];
    const int t = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * kSumBlock;
    buf[t] = base + t < n ? x[base + t] : 0.0;
    buf[t + kSumBlock / 2] = base + t + kSumBlock / 2 < n ? x[base + t + kSumBlock / 2] : 0.0;
    __syncthreads();
    for (int s = kSumBlock / 2; s >= 1; s >>= 1) {
        if (t < s) buf[t] = __dadd_rn(buf[t], buf[t + s]);
        __syncthreads();
    }
    if (t == 0) out[blockIdx.x] = buf[0];
}

__global__ void k_graph_validate(int64_t n_nodes, int64_t n_arcs, const int32_t* __restrict__ src,
                                 const int32_t* __restrict__ dst, const float* __restrict__ w,
                                 uint32_t* status) {
    bool bad = false;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_arcs;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = src[e], d = dst[e];
        bad |= s < 0 || s >= n_nodes || d < 0 || d >= n_nodes;
        if (e > 0) bad |= src[e - 1] > s;
        if (w) {
            const float x = w[e];
            bad |= !(x > 0.0f) || !isfinite(x);
        }
    }
    if (bad) atomicOr(status, DEV_ERR_GRAPH);
}

__global__ void k_edge_weights(int64_t n, const float* __restrict__ w, double* __restrict__ x) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        x[e] = w ? (double)w[e] : 1.0;
}

__device__ __forceinline__ void store_neg_weight(double d, int64_t v, double* __restrict__ x, float* __restrict__ deg) {
    double r = 0.0;
    if (d > 0.0) {
        const double s = __dsqrt_rn(d);
        r = __dmul_rn(s, __dsqrt_rn(s));
    }
    x[v] = r;
    if (deg) deg[v] = (float)d;
}

// flag != 0 when some arc weight is not an integer in [1, 2^24].
__global__ void k_weights_integral(int64_t n, const float* __restrict__ w, uint32_t* flag) {
    bool bad = false;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float v = w[e];
        bad |= !(v >= 1.0f && v <= 16777216.0f && v == truncf(v));
    }
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// x_v = d(v)^0.75 = sqrt(d) * sqrt(sqrt(d)), d = weights of v's arcs summed in
// arc order (src is sorted, so v's arcs are the range row_ptr[v] ..
// row_ptr[v+1]).  Integer weights (flag == 0): a warp takes 32 consecutive
// nodes, sums each node's weights across its lanes in 64-bit integers -
// exact, so equal to the FP64 sum in arc order (partial sums stay below
// 2^53) - and lane k keeps node k's sum; then every lane takes the FP64
// square roots of its own node.  GB300's FP64 pipe is slow: the weights
// (integers in [1, 2^24]) are converted through 32-bit integers, and the
// FP64 work is one root pair per node on full warps.
__global__ void k_neg_weights_int(int64_t n_nodes, const int64_t* __restrict__ row_ptr,
                                  const float* __restrict__ w, const uint32_t* flag, double* __restrict__ x,
                                  float* __restrict__ deg) {
    if (flag && *flag) return;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t v0 = 32 * (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)); v0 < n_nodes;
         v0 += 32 * warps) {
        // lane k: the arc range of node v0 + k
        const int64_t vl = v0 + lane;
        const int64_t lo_l = vl < n_nodes ? row_ptr[vl] : 0, hi_l = vl < n_nodes ? row_ptr[vl + 1] : 0;
        unsigned long long mine = 0;
        if (w) {
            const int64_t nk = min((int64_t)32, n_nodes - v0);
            for (int k = 0; k < nk; ++k) {
                const int64_t lo = __shfl_sync(0xFFFFFFFFu, lo_l, k), hi = __shfl_sync(0xFFFFFFFFu, hi_l, k);
                unsigned long long sum = 0;
                for (int64_t e = lo + lane; e < hi; e += 32) sum += __float2uint_rz(w[e]);
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
                if (lane == k) mine = sum;
            }
        } else {
            mine = (unsigned long long)(hi_l - lo_l);
        }
        if (vl < n_nodes) store_neg_weight((double)mine, vl, x, deg);
    }
}

// Any other weights (flag != 0): one thread per node adds them in FP64 in arc
// order.
__global__ void k_neg_weights(int64_t n_nodes, const int64_t* __restrict__ row_ptr,
                              const float* __restrict__ w, const uint32_t* flag, double* __restrict__ x,
                              float* __restrict__ deg) {
    if (!*flag) return;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_nodes;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = row_ptr[v], hi = row_ptr[v + 1];
        double d = 0.0;
        for (int64_t e = lo; e < hi; ++e) d = __dadd_rn(d, (double)w[e]);
        store_neg_weight(d, v, x, deg);
    }
}

struct MassCounters {
    unsigned long long sum_m;  // sum of floor(x_i S)
    unsigned long long npos;   // #(x_i > 0)
    unsigned long long nge1;   // #(m_i >= 1)
    unsigned long long pad;
};

// m_i = floor(x_i * S), S = (n * 2^32) / W.
__global__ void k_masses(int64_t n, const double* __restrict__ x, const double* __restrict__ W,
                         uint64_t* __restrict__ m, MassCounters* cnt, uint32_t* status) {
    const double w = *W;
    if (!(w > 0.0) || !isfinite(w)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, DEV_ERR_ALIAS);
        return;
    }
    const double S = __ddiv_rn(__dmul_rn((double)n, 4294967296.0), w);
    unsigned long long sm = 0, np = 0, ng = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double xi = x[i];
        const uint64_t mi = (uint64_t)floor(__dmul_rn(xi, S));
        m[i] = mi;
        sm += mi;
        np += xi > 0.0;
        ng += mi >= 1;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sm += __shfl_xor_sync(0xFFFFFFFFu, sm, o);
        np += __shfl_xor_sync(0xFFFFFFFFu, np, o);
        ng += __shfl_xor_sync(0xFFFFFFFFu, ng, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&cnt->sum_m, sm);
        atomicAdd(&cnt->npos, np);
        atomicAdd(&cnt->nge1, ng);
    }
}

struct GenPos {
    const double* x;
    __device__ uint32_t operator()(int64_t i) const { return x[i] > 0.0 ? 1u : 0u; }
};
struct GenGe1 {
    const uint64_t* m;
    __device__ uint32_t operator()(int64_t i) const { return m[i] >= 1 ? 1u : 0u; }
};
// D > 0: q to every positive item, +1 more to the first r of them.
struct OutAddRR {
    const double* x;
    uint64_t* m;
    uint64_t q, r;
    __device__ void operator()(int64_t i, uint32_t excl, uint32_t) const {
        if (x[i] > 0.0) m[i] += q + ((uint64_t)excl < r ? 1ull : 0ull);
    }
};
// D < 0: -1 to the first |D| items with m >= 1.
struct OutSubFirst {
    uint64_t* m;
    uint64_t need;
    __device__ void operator()(int64_t i, uint32_t excl, uint32_t) const {
        if (m[i] >= 1 && (uint64_t)excl < need) m[i] -= 1;
    }
};

struct GenClass {
    const uint64_t* m;
    __device__ Quad operator()(int64_t i) const {
        const uint64_t v = m[i];
        if (v < kQ) return {1u, 0u, kQ - v, 0ull};
        if (v > kQ) return {0u, 1u, 0ull, v - kQ};
        return {0u, 0u, 0ull, 0ull};
    }
};
struct OutClass {
    const uint64_t* m;
    uint32_t* light_idx;
    uint64_t* dp;  // inclusive prefix of deficits, by light rank
    uint32_t* heavy_idx;
    uint64_t* ep;  // inclusive prefix of excesses, by heavy rank
    uint2* tab;
    __device__ void operator()(int64_t i, const Quad& excl, const Quad& incl) const {
        const uint64_t v = m[i];
        if (v < kQ) {
            light_idx[excl.a] = (uint32_t)i;
            dp[excl.a] = incl.c;
        } else if (v > kQ) {
            heavy_idx[excl.b] = (uint32_t)i;
            ep[excl.b] = incl.d;
        } else {
            tab[i] = make_uint2(kThrFull, (uint32_t)i);
        }
    }
};

__device__ __forceinline__ uint32_t lower_bound_u64(const uint64_t* a, uint32_t n, uint64_t v) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ uint32_t upper_bound_u64(const uint64_t* a, uint32_t n, uint64_t v) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_pair_lights(const Quad* total, const uint64_t* __restrict__ m, const uint32_t* __restrict__ light_idx,
                              const uint64_t* __restrict__ dp, const uint32_t* __restrict__ heavy_idx,
                              const uint64_t* __restrict__ ep, uint2* __restrict__ tab, uint32_t* status) {
    const uint32_t L = total->a, H = total->b;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < L; j += gridDim.x * blockDim.x) {
        const uint32_t i = light_idx[j];
        const uint64_t dpex = j ? dp[j - 1] : 0ull;
        const uint32_t k = lower_bound_u64(ep, H, dpex);
        if (k >= H) {
            atomicOr(status, DEV_ERR_ALIAS);
            continue;
        }
        tab[i] = make_uint2((uint32_t)m[i], heavy_idx[k]);
    }
}

__global__ void k_pair_heavies(const Quad* total, const uint64_t* __restrict__ dp, const uint32_t* __restrict__ heavy_idx,
                               const uint64_t* __restrict__ ep, uint2* __restrict__ tab, uint32_t* status) {
    const uint32_t L = total->a, H = total->b;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < H; k += gridDim.x * blockDim.x) {
        const uint32_t i = heavy_idx[k];
        if (k + 1 == H) {
            // the totals of deficits and excesses must agree exactly
            if (L == 0 || dp[L - 1] != ep[k]) atomicOr(status, DEV_ERR_ALIAS);
            tab[i] = make_uint2(kThrFull, i);
            continue;
        }
        const uint32_t j = upper_bound_u64(dp, L, ep[k]);
        if (j >= L || dp[j] - ep[k] > kQ) {
            atomicOr(status, DEV_ERR_ALIAS);
            continue;
        }
        tab[i] = make_uint2((uint32_t)(kQ - (dp[j] - ep[k])), heavy_idx[k + 1]);
    }
}

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 32) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

inline size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

size_t fixed_sum_tmp_bytes(int64_t n) {
    size_t total = 0;
    int64_t cur = n;
    do {
        cur = (cur + kSumBlock - 1) / kSumBlock;
        total += align_up(sizeof(double) * (size_t)(cur > 0 ? cur : 1));
    } while (cur > 1);
    return total;
}

cudaError_t fixed_sum_f64(const double* x, int64_t n, double* tmp, double* out, cudaStream_t s) {
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(double), s);
    const double* in = x;
    int64_t cur = n;
    char* p = (char*)tmp;
    while (true) {
        const int64_t nb = (cur + kSumBlock - 1) / kSumBlock;
        double* dst = nb == 1 ? out : (double*)p;
        k_tree_sum<<<(unsigned)nb, kSumBlock / 2, 0, s>>>(in, cur, dst);
        if (nb == 1) break;
        p += align_up(sizeof(double) * (size_t)nb);
        in = dst;
        cur = nb;
    }
    return cudaGetLastError();
}

cudaError_t validate_graph(int64_t n_nodes, int64_t n_arcs, const int32_t* src, const int32_t* dst, const float* w,
                           uint32_t* status, cudaStream_t s) {
    k_graph_validate<<<grid_for(n_arcs, 256), 256, 0, s>>>(n_nodes, n_arcs, src, dst, w, status);
    return cudaGetLastError();
}

cudaError_t edge_weights(int64_t n_arcs, const float* w, double* x, cudaStream_t s) {
    k_edge_weights<<<grid_for(n_arcs, 256), 256, 0, s>>>(n_arcs, w, x);
    return cudaGetLastError();
}

cudaError_t neg_weights(int64_t n_nodes, int64_t n_arcs, const int64_t* row_ptr, const float* w, double* x, float* deg,
                        uint32_t* flag, cudaStream_t s) {
    if (!w) {  // unit weights: the arc counts
        k_neg_weights_int<<<grid_for(n_nodes, 256, 152 * 16), 256, 0, s>>>(n_nodes, row_ptr, w, nullptr, x, deg);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_weights_integral<<<grid_for(n_arcs, 256, 152 * 32), 256, 0, s>>>(n_arcs, w, flag);
    k_neg_weights_int<<<grid_for(n_nodes, 256, 152 * 16), 256, 0, s>>>(n_nodes, row_ptr, w, flag, x, deg);
    k_neg_weights<<<grid_for(n_nodes, 128, 1 << 20), 128, 0, s>>>(n_nodes, row_ptr, w, flag, x, deg);
    return cudaGetLastError();
}

// tmp layout: W | counters | m[n] | dp[n] | ep[n] | light_idx[n] | heavy_idx[n] |
//             scan tiles (u32) | scan tiles (Quad) | fixed-sum tmp
size_t alias_build_tmp_bytes(int64_t n) {
    const int64_t nt = scan_tiles(n) + 1;
    return align_up(sizeof(double)) + align_up(sizeof(MassCounters)) + 3 * align_up(sizeof(uint64_t) * n) +
           2 * align_up(sizeof(uint32_t) * n) + align_up(sizeof(uint32_t) * nt) + align_up(sizeof(Quad) * nt) +
           fixed_sum_tmp_bytes(n);
}

cudaError_t alias_build(const double* x, int64_t n, uint2* tab, void* tmp, uint32_t* status, cudaStream_t s) {
    char* p = (char*)tmp;
    auto take = [&](size_t bytes) {
        char* r = p;
        p += align_up(bytes);
        return (void*)r;
    };
    double* W = (double*)take(sizeof(double));
    MassCounters* cnt = (MassCounters*)take(sizeof(MassCounters));
    uint64_t* m = (uint64_t*)take(sizeof(uint64_t) * n);
    uint64_t* dp = (uint64_t*)take(sizeof(uint64_t) * n);
    uint64_t* ep = (uint64_t*)take(sizeof(uint64_t) * n);
    uint32_t* light_idx = (uint32_t*)take(sizeof(uint32_t) * n);
    uint32_t* heavy_idx = (uint32_t*)take(sizeof(uint32_t) * n);
    const int64_t nt = scan_tiles(n) + 1;
    uint32_t* tiles32 = (uint32_t*)take(sizeof(uint32_t) * nt);
    Quad* tilesQ = (Quad*)take(sizeof(Quad) * nt);
    double* sum_tmp = (double*)p;

    cudaError_t e;
    if ((e = fixed_sum_f64(x, n, sum_tmp, W, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(MassCounters), s)) != cudaSuccess) return e;
    k_masses<<<grid_for(n, 256), 256, 0, s>>>(n, x, W, m, cnt, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    MassCounters h;
    if ((e = cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    const uint64_t target = (uint64_t)n * kQ;
    const int64_t D = (int64_t)(target - (uint64_t)h.sum_m);
    if (D > 0) {
        if (h.npos == 0) {
            uint32_t bit = DEV_ERR_ALIAS;
            return cudaMemcpyAsync(status, &bit, sizeof(bit), cudaMemcpyHostToDevice, s);
        }
        OutAddRR out{x, m, (uint64_t)D / h.npos, (uint64_t)D % h.npos};
        if ((e = device_scan<uint32_t>(n, GenPos{x}, out, tiles32, s)) != cudaSuccess) return e;
    } else if (D < 0) {
        if ((uint64_t)(-D) > h.nge1) {
            uint32_t bit = DEV_ERR_ALIAS;
            return cudaMemcpyAsync(status, &bit, sizeof(bit), cudaMemcpyHostToDevice, s);
        }
        OutSubFirst out{m, (uint64_t)(-D)};
        if ((e = device_scan<uint32_t>(n, GenGe1{m}, out, tiles32, s)) != cudaSuccess) return e;
    }
    OutClass oc{m, light_idx, dp, heavy_idx, ep, tab};
    if ((e = device_scan<Quad>(n, GenClass{m}, oc, tilesQ, s)) != cudaSuccess) return e;
    const Quad* total = tilesQ + (nt - 1);
    k_pair_lights<<<grid_for(n, 256), 256, 0, s>>>(total, m, light_idx, dp, heavy_idx, ep, tab, status);
    k_pair_heavies<<<grid_for(n, 256), 256, 0, s>>>(total, dp, heavy_idx, ep, tab, status);
    return cudaGetLastError();
}

}  // namespace line
