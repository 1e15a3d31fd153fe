// Warm start of new or held-out nodes: a two-layer MLP regresses a node's
// trained U row on its log weighted degree and the mean trained U row of its
// neighbours; its predictions initialise the rows of nodes LINE never
// trained (Algorithm 1 starts every row from a random draw), after which
// plain LINE refinement continues.
//
//   x = [log(1 + d_w(v)), mean_{v->w, w known} U[w], 0 pad]   (P = round16(d+1))
//   a = W1 x + b1,  h = GELU(a) = a/2 (1 + erf(a/sqrt 2)),  y = W2 h + b2
//   L = sum (y - U[v])^2 / (B d) over a minibatch,  Adam (beta 0.9/0.999, eps 1e-8)
//
// Weights, gradients and optimiser state are FP32; the activations x and h
// are stored as FP32 or BF16 (round to nearest even).  With FP32 activations
// every contraction is one tiled kernel with FP32 FMA accumulation in index
// order (split over the batch into slices summed in slice order for the
// weight gradients).  With BF16 activations the contractions run on the
// tensor cores in mlp_fwd.cu: the forward products and dL/da against the
// weights' BF16 hi/lo pairs, the weight gradients with dL/dy and dL/da as
// BF16 hi/lo pairs (k_gemm_tc, TF32, takes shapes those kernels do not).
// Either way every sum has a fixed order, so training is bitwise
// reproducible.  Random numbers: Philox domain 7, call 0
// for minibatch picks (counter s*B + j), call 1 for the initial weights
// (counter = the parameter's flat index).
#include <math.h>

#include <algorithm>
#include <atomic>
#include <type_traits>
#include <vector>

#include "context.cuh"
#include "mlp_fwd.cuh"
#include "mlp_math.cuh"

namespace line {

constexpr uint32_t kMlpDomain = 7;
constexpr int64_t kMlpMaxBatch = 1 << 16;

struct MlpState {
    int order = 0, dim = 0, hidden = 0, P = 0, act = 0;
    int64_t n_params = 0;
    float* params = nullptr;  // [W1 (hidden x P) | b1 (hidden) | W2 (dim x hidden) | b2 (dim)];
                              // grads, m and v follow in the same allocation
    float* grads = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    int64_t t = 0;  // Adam steps taken
    void* X = nullptr;  // [n_nodes][P] features (act dtype)
    int64_t n_nodes = 0;
    bool has_features = false;
    // minibatch scratch (cap rows)
    int64_t cap = 0;
    int32_t* rows = nullptr;
    void* Xb = nullptr;      // [cap][P]
    float* Tb = nullptr;     // [cap][dim]
    float* A1 = nullptr;     // [cap][hidden] pre-activations
    void* Hb = nullptr;      // [cap][hidden] activations
    float* Yb = nullptr;     // [cap][dim] outputs, then dL/dy
    float* dH = nullptr;     // [cap][hidden] dL/dh, then dL/da
    // BF16 hi/lo pairs of dL/dy ([2][cap][dim]) and dL/da ([2][cap][hidden]),
    // the first operands of the tensor-core weight gradients
    __nv_bfloat16* gY = nullptr;
    __nv_bfloat16* gA = nullptr;
    void* arena = nullptr;  // the allocation holding every batch buffer above
    float* part = nullptr;   // split partials
    size_t part_elems = 0;
    double* rowloss = nullptr;  // [cap]
    void* sum_tmp = nullptr;
    double* losses = nullptr;   // [loss_cap] per-step losses
    int64_t loss_cap = 0;
    int32_t* nodes = nullptr;   // training node list (device copy)
    int64_t nodes_cap = 0;
    // input computation scratch: the known mask, the hub list ([count] then
    // ids), the requested rows and their range flag
    uint8_t* kmask = nullptr;
    uint32_t* hubs = nullptr;
    int64_t hubs_cap = 0;
    int32_t* frows = nullptr;
    int64_t frows_cap = 0;
    uint32_t* flag = nullptr;
    // the weights as tensor-core tiles (TF32, core-matrix layout), rebuilt by
    // every forward pass: W1 and W2 as the B operands of the forward
    // products, W2 as that of dL/dh
    float* wt = nullptr;
    size_t wt_elems = 0;
    // BF16 hi/lo tiles of W1 and W2 for the forward products of mlp_fwd.cu
    __nv_bfloat16* w16 = nullptr;
    size_t w16_elems = 0;
};

void mlp_destroy(MlpState* s) {
    if (!s) return;
    // params, grads, m and v share one allocation (params first); the
    // batch buffers share s->arena
    for (void* p : {(void*)s->params, s->X, s->arena, (void*)s->losses, (void*)s->nodes, (void*)s->kmask,
                    (void*)s->hubs, (void*)s->frows, (void*)s->flag, (void*)s->wt, (void*)s->w16})
        if (p) cudaFree(p);
    delete s;
}

namespace {

// ---- element helpers -------------------------------------------------------
template <typename T>
__device__ __forceinline__ float to_f(T x);
template <>
__device__ __forceinline__ float to_f<float>(float x) { return x; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename T>
__device__ __forceinline__ T from_f(float x);
template <>
__device__ __forceinline__ float from_f<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }


__device__ __forceinline__ float load_row_elem(const void* U, int dtype, int64_t idx) {
    return dtype == LINE_DTYPE_F32 ? reinterpret_cast<const float*>(U)[idx]
                                   : __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(U)[idx]);
}


// ---- initialisation --------------------------------------------------------
__global__ void k_mlp_init(float* __restrict__ p, int H, int P, int D, uint64_t seed, float s1, float s2) {
    const int64_t n1 = (int64_t)H * P, n2 = (int64_t)D * H;
    const int64_t total = n1 + H + n2 + D;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const uint4 w = draw_words(seed, kMlpDomain, (uint64_t)t, 1u);
        const float u = (float)((int32_t)(w.x >> 8) - (1 << 23)) * (1.0f / 8388608.0f);
        float val = 0.0f;
        if (t < n1) {
            if ((int)(t % P) <= D) val = u * s1;
        } else if (t >= n1 + H && t < n1 + H + n2) {
            val = u * s2;
        }
        p[t] = val;
    }
}

// ---- features: one warp per node -------------------------------------------
// Nodes with more than kHubArcs arcs ("hubs") are summed by CTAs of
// kHubWarps warps, one CTA per chunk of kHubChunk arcs: a hub of hundreds of
// thousands of arcs is spread over many SMs instead of holding one.
constexpr int64_t kHubArcs = 256;
constexpr int64_t kHubChunk = 2048;
constexpr int kHubWarps = 16;
constexpr int kPlanThreads = 1024;

// Hub-path scratch for a graph of n_nodes nodes and n_arcs arcs: a bitmap
// of the hubs already listed (a node requested twice is listed once), the
// hub count and list, the chunk offsets of all hubs and of the hubs with
// two or more chunks (whose chunk sums are combined afterwards), and those
// chunk sums.  At most n_arcs / kHubArcs distinct nodes are hubs; a hub of
// more than kHubChunk arcs has fewer than 2 deg / kHubChunk chunks, so the
// multi-chunk hubs have fewer than 2 n_arcs / kHubChunk chunks in all.
struct HubScratch {
    int64_t max_hubs, max_multi, map_words;
    HubScratch(int64_t n_nodes, int64_t n_arcs)
        : max_hubs(n_arcs / kHubArcs + 1), max_multi(2 * n_arcs / kHubChunk + 1), map_words((n_nodes + 31) / 32) {}
    size_t list_words() const { return (size_t)max_hubs + 1; }
    size_t off_words() const { return (size_t)max_hubs + 1; }
    size_t bytes(int D) const {
        return sizeof(uint32_t) * ((size_t)map_words + list_words() + 2 * off_words() + (size_t)max_multi) +
               sizeof(float) * (size_t)max_multi * D + 256;
    }
};

// Row geometry of the inputs: lane l holds values [l E, l E + E) of a row of
// D values (E = D/32, or 1 with lanes >= D idle when D < 32), loaded as one
// vector.
template <int D>
struct FGeom {
    static constexpr int E = D >= 32 ? D / 32 : 1;
    static constexpr int LANES = D / E;
};

template <int D, int UDT>
__device__ __forceinline__ void load_vals(const void* U, int64_t row, int lane, float (&v)[FGeom<D>::E]) {
    constexpr int E = FGeom<D>::E;
    if constexpr (UDT == LINE_DTYPE_F32) {
        const float* p = reinterpret_cast<const float*>(U) + row * D + lane * E;
        if constexpr (E == 8) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p) + 1);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else if constexpr (E == 4) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(p));
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        } else if constexpr (E == 2) {
            const float2 a = __ldg(reinterpret_cast<const float2*>(p));
            v[0] = a.x; v[1] = a.y;
        } else {
            v[0] = __ldg(p);
        }
    } else {
        const __nv_bfloat16* p = reinterpret_cast<const __nv_bfloat16*>(U) + row * D + lane * E;
        if constexpr (E == 8) {
            const uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
            const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                v[2 * i] = __uint_as_float(w[i] << 16);
                v[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
            }
        } else if constexpr (E == 4) {
            const uint2 a = __ldg(reinterpret_cast<const uint2*>(p));
            v[0] = __uint_as_float(a.x << 16); v[1] = __uint_as_float(a.x & 0xFFFF0000u);
            v[2] = __uint_as_float(a.y << 16); v[3] = __uint_as_float(a.y & 0xFFFF0000u);
        } else if constexpr (E == 2) {
            const uint32_t a = __ldg(reinterpret_cast<const unsigned int*>(p));
            v[0] = __uint_as_float(a << 16); v[1] = __uint_as_float(a & 0xFFFF0000u);
        } else {
            v[0] = __bfloat162float(p[0]);
        }
    }
}

// Adds the rows U[dst[e]] of the known neighbours among arcs [lo, hi) to acc
// in arc order (each value's sum runs over the neighbours in arc order);
// returns their number.  Arcs are taken 32 at a time (one per lane), and up
// to 8 known rows (4 at d = 256) are loaded at once before they are added.
template <int D, int UDT>
__device__ __forceinline__ int sum_known_rows(int64_t lo, int64_t hi, const int32_t* __restrict__ dst, const void* U,
                                             const uint8_t* __restrict__ known, float (&acc)[FGeom<D>::E]) {
    using F = FGeom<D>;
    constexpr int kGroup = F::E <= 4 ? 8 : 4;
    const int lane = threadIdx.x & 31;
    const bool holds = lane < F::LANES;
    int cnt = 0;
    for (int64_t e0 = lo; e0 < hi; e0 += 32) {
        const int64_t e = e0 + lane;
        const int32_t w = e < hi ? __ldg(dst + e) : 0;
        const bool ok = e < hi && __ldg(known + w);
        uint32_t mask = __ballot_sync(0xFFFFFFFFu, ok);
        cnt += __popc(mask);
        while (mask) {
            int32_t rows[kGroup];
            int m = 0;
#pragma unroll
            for (int j = 0; j < kGroup; ++j) {
                rows[j] = 0;
                if (mask) {
                    const int l = __ffs(mask) - 1;
                    mask &= mask - 1;
                    rows[j] = __shfl_sync(0xFFFFFFFFu, w, l);
                    m = j + 1;
                }
            }
            float val[kGroup][F::E];
#pragma unroll
            for (int j = 0; j < kGroup; ++j)
                if (j < m && holds) load_vals<D, UDT>(U, rows[j], lane, val[j]);
#pragma unroll
            for (int j = 0; j < kGroup; ++j)
                if (j < m)
#pragma unroll
                    for (int i = 0; i < F::E; ++i) acc[i] += val[j][i];
        }
    }
    return cnt;
}

template <int D, typename TX>
__device__ __forceinline__ void write_features(TX* x, float deg, const float (&acc)[FGeom<D>::E], int cnt, int P) {
    using F = FGeom<D>;
    const int lane = threadIdx.x & 31;
    if (lane == 0) x[0] = from_f<TX>(log1pf(deg));
    if (lane < F::LANES) {
#pragma unroll
        for (int i = 0; i < F::E; ++i) x[1 + lane * F::E + i] = from_f<TX>(cnt ? acc[i] / (float)cnt : 0.0f);
    }
    for (int k = D + 1 + lane; k < P; k += 32) x[k] = from_f<TX>(0.0f);
}

// flag |= 1 if a requested row id is out of range.
__global__ void k_check_rows(const int32_t* __restrict__ rows, int64_t n_rows, int64_t n_nodes, uint32_t* flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_rows; i += (int64_t)gridDim.x * blockDim.x)
        if (rows[i] < 0 || rows[i] >= n_nodes) atomicOr(flag, 1u);
}

struct FeatParams {
    int64_t n_nodes;
    const int64_t* row_ptr;
    const int32_t* dst;
    const float* deg;
    const void* U;
    const uint8_t* known;
    int P;
    void* X;
    uint32_t* hub_map;  // [n_nodes / 32] bit v: node v is listed (zero at the call's start)
    uint32_t* hubs;     // listed hub nodes
    uint32_t* n_hubs;   // their number
    uint32_t* off;     // [n_hubs + 1] first chunk of each hub (all hubs)
    uint32_t* poff;    // [n_hubs + 1] first chunk-sum slot of each multi-chunk hub
    float* part;       // [slots][D] chunk sums of the multi-chunk hubs
    uint32_t* pcnt;    // [slots] their known-neighbour counts
    const int32_t* rows;
    int64_t n_rows;
    const uint32_t* flag;
};

// One warp per node; nodes with more than kHubArcs arcs are listed in hubs
// (order irrelevant) and left to k_mlp_features_hub.  Nothing is written
// when *flag is set (a requested row id was out of range).
template <int D, int UDT, typename TX>
__global__ void __launch_bounds__(256, 3) k_mlp_features(FeatParams p) {
    if (*(volatile const uint32_t*)p.flag) return;
    using F = FGeom<D>;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t count = p.rows ? p.n_rows : p.n_nodes;
    for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < count; r += warps) {
        const int64_t v = p.rows ? (int64_t)p.rows[r] : r;
        const int64_t lo = __ldg(p.row_ptr + v), hi = __ldg(p.row_ptr + v + 1);
        if (hi - lo > kHubArcs) {
            if (lane == 0) {
                const uint32_t bit = 1u << (v & 31);
                if (!(atomicOr(p.hub_map + (v >> 5), bit) & bit)) p.hubs[atomicAdd(p.n_hubs, 1u)] = (uint32_t)v;
            }
            continue;
        }
        float acc[F::E];
#pragma unroll
        for (int i = 0; i < F::E; ++i) acc[i] = 0.0f;
        const int cnt = sum_known_rows<D, UDT>(lo, hi, p.dst, p.U, p.known, acc);
        write_features<D, TX>(reinterpret_cast<TX*>(p.X) + v * (int64_t)p.P, __ldg(p.deg + v), acc, cnt, p.P);
    }
}

__device__ __forceinline__ uint32_t hub_chunks(const FeatParams& p, uint32_t h) {
    const int64_t v = p.hubs[h];
    return (uint32_t)((p.row_ptr[v + 1] - p.row_ptr[v] + kHubChunk - 1) / kHubChunk);
}

// One CTA: the exclusive prefix sums, in listing order, of the hubs' chunk
// counts (off) and of the chunk counts of the hubs with two or more chunks
// (poff); off[n] and poff[n] are the totals.
__global__ void __launch_bounds__(kPlanThreads) k_hub_plan(FeatParams p) {
    __shared__ uint32_t wsum[2][kPlanThreads / 32];
    __shared__ uint32_t carry[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nh = *p.n_hubs;
    if (threadIdx.x < 2) carry[threadIdx.x] = 0u;
    __syncthreads();
    for (uint32_t base = 0; base < nh; base += kPlanThreads) {
        const uint32_t h = base + threadIdx.x;
        const uint32_t c = h < nh ? hub_chunks(p, h) : 0u;
        uint32_t x[2] = {c, c > 1 ? c : 0u};
        // inclusive warp scans, then the warp totals scanned by warp 0
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x[k], o);
                if (lane >= o) x[k] += y;
            }
        if (lane == 31) {
            wsum[0][warp] = x[0];
            wsum[1][warp] = x[1];
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                uint32_t t = wsum[k][lane];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
                    if (lane >= o) t += y;
                }
                wsum[k][lane] = t;  // inclusive over warps
            }
        }
        __syncthreads();
        if (h < nh) {
            const uint32_t before0 = warp ? wsum[0][warp - 1] : 0u, before1 = warp ? wsum[1][warp - 1] : 0u;
            p.off[h] = carry[0] + before0 + x[0] - c;
            p.poff[h] = carry[1] + before1 + x[1] - (c > 1 ? c : 0u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry[0] += wsum[0][kPlanThreads / 32 - 1];
            carry[1] += wsum[1][kPlanThreads / 32 - 1];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        p.off[nh] = carry[0];
        p.poff[nh] = carry[1];
    }
}

// Chunk i of the hubs' arcs (hub h = the last with off[h] <= i, chunk
// c = i - off[h] of kHubChunk arcs): warp w sums the w-th of kHubWarps
// contiguous slices of the chunk, the warps' sums are added in warp order;
// a one-chunk hub's inputs are written at once, the other chunks' sums go
// to their slots for k_hub_combine.
template <int D, int UDT, typename TX>
__global__ void __launch_bounds__(kHubWarps * 32) k_mlp_features_hub(FeatParams p) {
    using F = FGeom<D>;
    __shared__ float part[kHubWarps][D];
    __shared__ int pcnt[kHubWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nh = *p.n_hubs;
    const uint32_t total = p.off[nh];
    for (uint32_t i = blockIdx.x; i < total; i += gridDim.x) {
        uint32_t lo_h = 0, hi_h = nh;  // off[lo_h] <= i < off[hi_h]
        while (hi_h - lo_h > 1) {
            const uint32_t mid = (lo_h + hi_h) >> 1;
            if (p.off[mid] <= i) lo_h = mid;
            else hi_h = mid;
        }
        const uint32_t h = lo_h, c = i - p.off[h];
        const int64_t v = p.hubs[h];
        const int64_t vlo = p.row_ptr[v], vhi = p.row_ptr[v + 1];
        const int64_t clo = vlo + (int64_t)c * kHubChunk, chi = min(vhi, clo + kHubChunk);
        const int64_t per = (chi - clo + kHubWarps - 1) / kHubWarps;
        const int64_t a = min(chi, clo + warp * per), b = min(chi, a + per);
        float acc[F::E];
#pragma unroll
        for (int k = 0; k < F::E; ++k) acc[k] = 0.0f;
        const int cw = sum_known_rows<D, UDT>(a, b, p.dst, p.U, p.known, acc);
        if (lane < F::LANES)
#pragma unroll
            for (int k = 0; k < F::E; ++k) part[warp][lane * F::E + k] = acc[k];
        if (lane == 0) pcnt[warp] = cw;
        __syncthreads();
        if (warp == 0) {
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < F::E; ++k) acc[k] = 0.0f;
            for (int w = 0; w < kHubWarps; ++w) {
                cnt += pcnt[w];
                if (lane < F::LANES)
#pragma unroll
                    for (int k = 0; k < F::E; ++k) acc[k] += part[w][lane * F::E + k];
            }
            if (vhi - vlo <= kHubChunk) {
                write_features<D, TX>(reinterpret_cast<TX*>(p.X) + v * (int64_t)p.P, p.deg[v], acc, cnt, p.P);
            } else {
                const uint32_t slot = p.poff[h] + c;
                if (lane < F::LANES)
#pragma unroll
                    for (int k = 0; k < F::E; ++k) p.part[(size_t)slot * D + lane * F::E + k] = acc[k];
                if (lane == 0) p.pcnt[slot] = (uint32_t)cnt;
            }
        }
        __syncthreads();
    }
}

// One warp per hub with two or more chunks: its chunk sums added in chunk
// order, then its inputs written.
template <int D, typename TX>
__global__ void k_hub_combine(FeatParams p) {
    using F = FGeom<D>;
    const int lane = threadIdx.x & 31;
    const uint32_t nh = *p.n_hubs;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t h = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); h < nh; h += warps) {
        const uint32_t c0 = p.poff[h], c1 = p.poff[h + 1];
        if (c1 == c0) continue;  // one chunk: written by k_mlp_features_hub
        float acc[F::E];
#pragma unroll
        for (int k = 0; k < F::E; ++k) acc[k] = 0.0f;
        int cnt = 0;
        for (uint32_t c = c0; c < c1; ++c) {
            cnt += (int)p.pcnt[c];
            if (lane < F::LANES)
#pragma unroll
                for (int k = 0; k < F::E; ++k) acc[k] += p.part[(size_t)c * D + lane * F::E + k];
        }
        const int64_t v = p.hubs[h];
        write_features<D, TX>(reinterpret_cast<TX*>(p.X) + v * (int64_t)p.P, p.deg[v], acc, cnt, p.P);
    }
}

template <int D, int UDT, typename TX>
cudaError_t launch_features(const FeatParams& p, int64_t count, int64_t max_hubs, cudaStream_t s) {
    const unsigned g = (unsigned)std::min<int64_t>((count + 7) / 8, 152 * 16);
    k_mlp_features<D, UDT, TX><<<g, 256, 0, s>>>(p);
    k_hub_plan<<<1, kPlanThreads, 0, s>>>(p);
    k_mlp_features_hub<D, UDT, TX><<<152 * 4, kHubWarps * 32, 0, s>>>(p);
    k_hub_combine<D, TX><<<(unsigned)std::min<int64_t>((max_hubs + 7) / 8, 152 * 4), 256, 0, s>>>(p);
    return cudaGetLastError();
}

template <int UDT, typename TX>
cudaError_t features_for(int D, const FeatParams& p, int64_t count, int64_t max_hubs, cudaStream_t s) {
    switch (D) {
        case 16: return launch_features<16, UDT, TX>(p, count, max_hubs, s);
        case 32: return launch_features<32, UDT, TX>(p, count, max_hubs, s);
        case 64: return launch_features<64, UDT, TX>(p, count, max_hubs, s);
        case 128: return launch_features<128, UDT, TX>(p, count, max_hubs, s);
        case 256: return launch_features<256, UDT, TX>(p, count, max_hubs, s);
        default: return cudaErrorInvalidValue;
    }
}

// ---- minibatch: rows[j] = nodes[mulhi64(w1:w0, n)], draw s*B + j ------------
__global__ void k_mlp_batch(const int32_t* __restrict__ nodes, int64_t n, uint64_t seed, uint64_t t0, int64_t B,
                            int32_t* __restrict__ rows) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < B; j += (int64_t)gridDim.x * blockDim.x) {
        const uint4 w = draw_words(seed, kMlpDomain, t0 + (uint64_t)j, 0u);
        const uint64_t r = ((uint64_t)w.y << 32) | (uint64_t)w.x;
        rows[j] = nodes[__umul64hi(r, (uint64_t)n)];
    }
}

// Xb[j] = X[rows[j]]; Tb[j] = U[rows[j]] (FP32) when Tb is given.
template <typename TX>
__global__ void k_mlp_gather(const int32_t* __restrict__ rows, int64_t B, int64_t n_nodes,
                             const TX* __restrict__ X, int P, TX* __restrict__ Xb, const void* U, int udt, int D,
                             float* __restrict__ Tb, uint32_t* status) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); j < B; j += warps) {
        int64_t r = rows[j];
        if (r < 0 || r >= n_nodes) {
            if (lane == 0) atomicOr(status, DEV_ERR_INDEX);
            r = 0;
        }
        for (int k = lane; k < P; k += 32) Xb[j * P + k] = X[r * P + k];
        if (Tb)
            for (int k = lane; k < D; k += 32) Tb[j * D + k] = load_row_elem(U, udt, r * D + k);
    }
}

// ---- the contraction -------------------------------------------------------
// C_z[m][n] = sum over k in slice z of A(m, k) B(k, n), k ascending;
// A(m, k) = AK ? A[m lda + k] : A[k lda + m], B(k, n) = BK ? B[n ldb + k] : B[k ldb + n].
constexpr int kBM = 64, kBN = 64, kBK = 16;

template <typename TA, typename TB, bool AK, bool BK>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, int kslice, const TA* __restrict__ A, int lda,
                                              const TB* __restrict__ B, int ldb, float* __restrict__ C) {
    __shared__ float As[kBK][kBM + 4];
    __shared__ float Bs[kBK][kBN + 4];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int kb = blockIdx.z * kslice, ke = min(K, kb + kslice);
    const int ty = tid / 16, tx = tid % 16;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int k0 = kb; k0 < ke; k0 += kBK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int mm = AK ? tid / 4 : (tid % 16) * 4 + q;
            const int ka = AK ? (tid % 4) * 4 + q : tid / 16;
            const int gm = m0 + mm, gk = k0 + ka;
            float a = 0.0f;
            if (gm < M && gk < ke) a = to_f(AK ? A[(size_t)gm * lda + gk] : A[(size_t)gk * lda + gm]);
            As[ka][mm] = a;
            const int nn = BK ? tid / 4 : (tid % 16) * 4 + q;
            const int kb2 = BK ? (tid % 4) * 4 + q : tid / 16;
            const int gn = n0 + nn, gk2 = k0 + kb2;
            float b = 0.0f;
            if (gn < N && gk2 < ke) b = to_f(BK ? B[(size_t)gn * ldb + gk2] : B[(size_t)gk2 * ldb + gn]);
            Bs[kb2][nn] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    float* Cz = C + (size_t)blockIdx.z * M * N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
            if (gm < M && gn < N) Cz[(size_t)gm * N + gn] = acc[i][j];
        }
}

// ---- the same contraction on the 5th-generation tensor cores (tcgen05) ----
// One CTA (8 warps) per 128 x NT tile of C (NT = 64, 128 or 256) and slice
// of K.  Per K step of 32 the threads stage A (128 x 32) and B (NT x 32) into
// shared memory as TF32 (rounded to nearest) in the no-swizzle K-major layout
// of 8-row x 16-byte core matrices (byte (r, k) = (r/8) 1024 + (k/4) 128 +
// (r%8) 16 + (k%4) 4).  Two stages: while the tensor core multiplies step i
// (one thread issues four tcgen05.mma kind::tf32 of K = 8 into a 128 x NT FP32
// tile in tensor memory and commits them to the stage's mbarrier), the
// threads stage step i+1 into the other buffers; a stage is refilled only
// after its previous MMAs completed.  Runs of 16 values contiguous in memory
// are loaded as vectors.  After the K loop warps w and w+4 read rows
// 32 (w%4) .. 32 (w%4) + 31 (their tensor-memory lanes), each half of the
// columns, with tcgen05.ld.  Every wait is bounded: on a timeout the tile is
// not written and the status word records it.
constexpr int kTcM = 128, kTcK = 32, kTcThreads = 256;
constexpr uint32_t kTcLbo = 128;                // next core matrix along K
constexpr uint32_t kTcSbo = (kTcK / 4) * 128;  // next group of 8 rows
constexpr int kTcWaitLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start >> 4, leading (K) byte offset >> 4,
// stride (8-row) byte offset >> 4, the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(kTcLbo >> 4) << 16) | ((uint64_t)(kTcSbo >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// 16 consecutive values of a row (T = float or BF16) at p; a vector load when
// aligned and complete, else element by element up to n.
template <typename T>
__device__ __forceinline__ void load16(const T* p, int n, float (&v)[16]) {
    if (n >= 16 && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 a = __ldg(reinterpret_cast<const float4*>(p) + q);
                v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const uint4 a = __ldg(reinterpret_cast<const uint4*>(p) + q);
                const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    v[8 * q + 2 * i] = __uint_as_float(w[i] << 16);
                    v[8 * q + 2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
                }
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = i < n ? to_f(p[i]) : 0.0f;
    }
}

// Stage rows [r0, r0 + R) x K step [k0, k0 + 32) of X (X(r, k) = XK ?
// X[r ld + k] : X[k ld + r]; values outside [0, rmax) x [k0, ke) are zero) as
// TF32 into the core-matrix layout at s.
template <typename T, bool XK, int R>
__device__ __forceinline__ void stage_tile(float* __restrict__ s, const T* __restrict__ X, int ld, int r0, int rmax,
                                           int k0, int ke) {
    if constexpr (XK) {
        // work item: (row, 16 consecutive k)
        for (int it = threadIdx.x; it < R * 2; it += kTcThreads) {
            const int r = it >> 1, kg = (it & 1) * 16;
            const int gr = r0 + r, gk = k0 + kg;
            float v[16];
            if (gr < rmax && gk < ke) load16(X + (size_t)gr * ld + gk, ke - gk, v);
            else
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float4* dst = reinterpret_cast<float4*>(s + (r >> 3) * (kTcSbo / 4) + ((kg >> 2) + q) * (kTcLbo / 4) + (r & 7) * 4);
                *dst = make_float4(to_tf32(v[4 * q]), to_tf32(v[4 * q + 1]), to_tf32(v[4 * q + 2]), to_tf32(v[4 * q + 3]));
            }
        }
    } else {
        // work item: (k, 16 consecutive rows)
        for (int it = threadIdx.x; it < (R / 16) * kTcK; it += kTcThreads) {
            const int k = it / (R / 16), rg = (it % (R / 16)) * 16;
            const int gk = k0 + k, gr = r0 + rg;
            float v[16];
            if (gk < ke && gr < rmax) load16(X + (size_t)gk * ld + gr, rmax - gr, v);
            else
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0.0f;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int r = rg + i;
                s[(r >> 3) * (kTcSbo / 4) + (k >> 2) * (kTcLbo / 4) + (r & 7) * 4 + (k & 3)] = to_tf32(v[i]);
            }
        }
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < kTcWaitLimit && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity));
    }
    return done != 0;
}

template <int NT>
constexpr size_t tc_smem_bytes() {
    return 1024 + 2 * sizeof(float) * (size_t)(kTcM + NT) * kTcK;  // 1024: room to align the stages
}

// Epilogue of the hidden layer (HID): C = A1 = acc + bias[n] and
// H[m][n] = GELU(A1) in TH, written straight from tensor memory.
template <typename TA, typename TB, bool AK, bool BK, int NT, bool HID = false, typename TH = float>
__global__ void __launch_bounds__(kTcThreads) k_gemm_tc(int M, int N, int K, int kslice, const TA* __restrict__ A,
                                                        int lda, const TB* __restrict__ B, int ldb,
                                                        const float* __restrict__ Bt, float* __restrict__ C,
                                                        uint32_t* status, const float* __restrict__ bias = nullptr,
                                                        TH* __restrict__ H = nullptr) {
    extern __shared__ unsigned char tc_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ __align__(8) uint64_t full[2];  // B tile of the stage arrived (bulk copy path)
    __shared__ uint32_t tmem_base;
    // stage st: A at base + st (128 x 32), B at base + 2 (128 x 32) + st (NT x 32)
    float* base = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kTcM, n0 = blockIdx.x * NT;
    const int kb = blockIdx.z * kslice, ke = min(K, kb + kslice);
    const int nk = ke > kb ? (ke - kb + kTcK - 1) / kTcK : 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[1])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    bool ok = true;
    for (int i = 0; i < nk; ++i) {
        const int st = i & 1;
        if (i >= 2) {
            // the MMAs of step i-2 read this stage
            ok = mbar_wait(smem_addr(&mbar[st]), (uint32_t)(((i - 2) >> 1) & 1));
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (!__syncthreads_and(ok)) break;
        }
        const int k0 = kb + i * kTcK;
        float* sa = base + st * (kTcM * kTcK);
        float* sb = base + 2 * (kTcM * kTcK) + st * (NT * kTcK);
        if (Bt) {
            // the B tile is already TF32 in the core-matrix layout: one bulk
            // copy, completing on the stage's `full` barrier
            if (tid == 0) {
                constexpr uint32_t bytes = NT * kTcK * sizeof(float);
                const float* src = Bt + ((size_t)blockIdx.x * ((K + kTcK - 1) / kTcK) + k0 / kTcK) * (NT * kTcK);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&full[st])),
                             "r"(bytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_addr(sb)),
                    "l"(src), "r"(bytes), "r"(smem_addr(&full[st]))
                    : "memory");
            }
        } else {
            stage_tile<TB, BK, NT>(sb, B, ldb, n0, N, k0, ke);
        }
        stage_tile<TA, AK, kTcM>(sa, A, lda, m0, M, k0, ke);
        asm volatile("fence.proxy.async.shared::cta;");  // the tensor core reads through the async proxy
        __syncthreads();
        bool issued = true;
        if (tid == 0) {
            if (Bt && !mbar_wait(smem_addr(&full[st]), (uint32_t)((i >> 1) & 1))) issued = false;
            asm volatile("tcgen05.fence::after_thread_sync;");
        }
        if (!__syncthreads_and(issued)) {
            ok = false;
            break;
        }
        if (tid == 0) {
#pragma unroll
            for (int kk = 0; kk < kTcK / 8; ++kk) {
                const uint64_t da = tc_smem_desc(smem_addr(sa) + kk * 2 * kTcLbo);
                const uint64_t db = tc_smem_desc(smem_addr(sb) + kk * 2 * kTcLbo);
                const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(tc_idesc(NT)), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&mbar[st])));
        }
    }
    if (ok && nk > 0) {
        // the last commit tracks every earlier MMA of this thread
        const int last = nk - 1;
        ok = mbar_wait(smem_addr(&mbar[last & 1]), (uint32_t)((last >> 1) & 1));
        asm volatile("tcgen05.fence::after_thread_sync;");
        ok = __syncthreads_and(ok);
    }
    float* Cz = C + (size_t)blockIdx.z * M * N;
    if (ok && nk > 0) {
        const int quarter = warp & 3, half = warp >> 2;
        const int row = m0 + quarter * 32 + lane;
#pragma unroll
        for (int c0 = half * (NT / 2); c0 < (half + 1) * (NT / 2); c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if constexpr (HID) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    r[j] = __float_as_uint(__uint_as_float(r[j]) + (n < N ? __ldg(bias + n) : 0.0f));
                }
                if (row < M) {
                    TH* hout = H + (size_t)row * N + n0 + c0;
                    if (n0 + c0 + 16 <= N && (reinterpret_cast<uintptr_t>(hout) & 15) == 0) {
                        if constexpr (sizeof(TH) == 2) {
                            uint32_t w[8];
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const __nv_bfloat162 v = __floats2bfloat162_rn(gelu(__uint_as_float(r[2 * q])),
                                                                               gelu(__uint_as_float(r[2 * q + 1])));
                                w[q] = *reinterpret_cast<const uint32_t*>(&v);
                            }
                            reinterpret_cast<uint4*>(hout)[0] = make_uint4(w[0], w[1], w[2], w[3]);
                            reinterpret_cast<uint4*>(hout)[1] = make_uint4(w[4], w[5], w[6], w[7]);
                        } else {
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                reinterpret_cast<float4*>(hout)[q] = make_float4(
                                    gelu(__uint_as_float(r[4 * q])), gelu(__uint_as_float(r[4 * q + 1])),
                                    gelu(__uint_as_float(r[4 * q + 2])), gelu(__uint_as_float(r[4 * q + 3])));
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (n0 + c0 + j < N) hout[j] = from_f<TH>(gelu(__uint_as_float(r[j])));
                    }
                }
            }
            if (row < M) {
                float* out = Cz + (size_t)row * N + n0 + c0;
                if (n0 + c0 + 16 <= N && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        reinterpret_cast<float4*>(out)[q] =
                            make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                        __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (n0 + c0 + j < N) out[j] = __uint_as_float(r[j]);
                }
            }
        }
    } else if (nk > 0) {
        if (tid == 0) atomicOr(status, DEV_ERR_TIMEOUT);
    } else {
        // an empty K slice: the partial sum is zero
        for (int i = tid; i < kTcM * NT; i += kTcThreads) {
            const int r = m0 + i / NT, cc = n0 + i % NT;
            if (r < M && cc < N) Cz[(size_t)r * N + cc] = 0.0f;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT));
}

template <typename TA, typename TB, bool AK, bool BK, int NT, bool HID = false, typename TH = float>
cudaError_t launch_tc(int M, int N, int K, int slices, const TA* A, int lda, const TB* B, int ldb, const float* Bt,
                      float* C, uint32_t* status, cudaStream_t s, const float* bias = nullptr, TH* H = nullptr) {
    constexpr size_t smem = tc_smem_bytes<NT>();
    static std::atomic<uint64_t> attr_set{0};  // devices whose kernel attribute is set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(attr_set.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(k_gemm_tc<TA, TB, AK, BK, NT, HID, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(bit, std::memory_order_acq_rel);
    }
    const int kslice = ((K + slices - 1) / slices + kTcK - 1) / kTcK * kTcK;
    const dim3 grid((N + NT - 1) / NT, (M + kTcM - 1) / kTcM, slices);
    k_gemm_tc<TA, TB, AK, BK, NT, HID, TH><<<grid, kTcThreads, smem, s>>>(M, N, K, kslice, A, lda, B, ldb, Bt, C,
                                                                           status, bias, H);
    return cudaGetLastError();
}

// The N tile of the tensor-core product: the widest that does not exceed N
// by more than half a tile.
inline int tc_tile_n(int N) { return N > 128 ? 256 : N > 64 ? 128 : 64; }

// Bt[(n_tile ceil(K/32) + k_step) NT 32 ...]: B(k, n) (BK ? B[n ldb + k] :
// B[k ldb + n]) as TF32 tiles of NT x 32 in the core-matrix layout of
// k_gemm_tc's stages, zero outside N x K.
template <bool BK>
__global__ void k_tile_b(const float* __restrict__ B, int ldb, int N, int K, int NT, float* __restrict__ Bt) {
    const int ks = (K + kTcK - 1) / kTcK, nt = (N + NT - 1) / NT;
    const int64_t total = (int64_t)nt * ks * NT * kTcK;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t tile = i / (NT * kTcK);
        const int r = (int)((i % (NT * kTcK)) / kTcK), k = (int)(i % kTcK);
        const int gn = (int)(tile / ks) * NT + r, gk = (int)(tile % ks) * kTcK + k;
        const float v = (gn < N && gk < K) ? (BK ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn]) : 0.0f;
        Bt[tile * (NT * kTcK) + (r >> 3) * (kTcSbo / 4) + (k >> 2) * (kTcLbo / 4) + (r & 7) * 4 + (k & 3)] = to_tf32(v);
    }
}

inline size_t tile_b_elems(int N, int K) {
    const int NT = tc_tile_n(N);
    return (size_t)((N + NT - 1) / NT) * ((K + kTcK - 1) / kTcK) * NT * kTcK;
}

// C_z = A B over K slice z, on the tensor cores when tc is set; Bt (tc only,
// nullable): B already as tiles (k_tile_b), copied in bulk.
template <typename TA, typename TB, bool AK, bool BK>
cudaError_t gemm(bool tc, int M, int N, int K, int slices, const TA* A, int lda, const TB* B, int ldb, float* C,
                 uint32_t* status, cudaStream_t s, const float* Bt = nullptr) {
    if (tc) {
        const int NT = tc_tile_n(N);
        if (NT == 256) return launch_tc<TA, TB, AK, BK, 256>(M, N, K, slices, A, lda, B, ldb, Bt, C, status, s);
        if (NT == 128) return launch_tc<TA, TB, AK, BK, 128>(M, N, K, slices, A, lda, B, ldb, Bt, C, status, s);
        return launch_tc<TA, TB, AK, BK, 64>(M, N, K, slices, A, lda, B, ldb, Bt, C, status, s);
    }
    const int kslice = ((K + slices - 1) / slices + kBK - 1) / kBK * kBK;
    const dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, slices);
    k_gemm<TA, TB, AK, BK><<<grid, 256, 0, s>>>(M, N, K, kslice, A, lda, B, ldb, C);
    return cudaGetLastError();
}

// ---- epilogues -------------------------------------------------------------
// A1 = A1 + b1 (in place), H = GELU(A1) in the activation type.
template <typename TH>
__global__ void k_ep_hidden(float* __restrict__ A1, const float* __restrict__ b1, int64_t M, int H, TH* __restrict__ Hb) {
    const int64_t n = M * H;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float a = A1[i] + b1[i % H];
        A1[i] = a;
        Hb[i] = from_f<TH>(gelu(a));
    }
}

// BF16 hi/lo pair of v at hl[i] and hl[half + i] (v = hi + lo to about 16
// significant bits).
__device__ __forceinline__ void store_hilo(__nv_bfloat16* hl, int64_t half, int64_t i, float v) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    hl[i] = hi;
    hl[half + i] = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// Training: y = Y + b2, r = y - t, dY = 2 r / (B D), rowloss[m] = sum r^2
// (FP32 per lane in column order, then over the lanes in butterfly order;
// the rows' sum is FP64).  One warp per row.  hl (nullable): dY's BF16
// hi/lo pair as well.
__global__ void k_ep_loss(float* __restrict__ Y, const float* __restrict__ b2, const float* __restrict__ Tb, int64_t M,
                          int D, float scale, double* __restrict__ rowloss, __nv_bfloat16* __restrict__ hl) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t m = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); m < M; m += warps) {
        float acc = 0.0f;
        for (int n = lane; n < D; n += 32) {
            const float r = (Y[m * D + n] + b2[n]) - Tb[m * D + n];
            acc = fmaf(r, r, acc);
            Y[m * D + n] = scale * r;
            if (hl) store_hilo(hl, M * D, m * D + n, scale * r);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) rowloss[m] = (double)acc;
    }
}

// Inference: y = Y + b2 into out[m] (FP32 rows) or, with rows, into table
// rows[m] of type `odt`.
__global__ void k_ep_predict(const float* __restrict__ Y, const float* __restrict__ b2, int64_t M, int D,
                             const int32_t* __restrict__ rows, int64_t n_nodes, void* out, int odt) {
    const int64_t n = M * D;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i / D, k = i - m * D;
        const float y = Y[i] + b2[k];
        if (rows && (rows[m] < 0 || rows[m] >= n_nodes)) continue;  // reported by the gather
        const int64_t dst = rows ? (int64_t)rows[m] * D + k : i;
        if (odt == LINE_DTYPE_F32) reinterpret_cast<float*>(out)[dst] = y;
        else reinterpret_cast<__nv_bfloat16*>(out)[dst] = __float2bfloat16_rn(y);
    }
}

// dA = dH * GELU'(A1), in place; hl (nullable): dA's BF16 hi/lo pair as well.
__global__ void k_ep_dact(float* __restrict__ dH, const float* __restrict__ A1, int64_t n,
                          __nv_bfloat16* __restrict__ hl) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = dH[i] * gelu_grad(A1[i]);
        dH[i] = v;
        if (hl) store_hilo(hl, n, i, v);
    }
}

// out[i] = sum_z part[z][i], z ascending.
__global__ void k_sum_slices(const float* __restrict__ part, int S, int64_t count, float* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
#pragma unroll 8
        for (int z = 0; z < S; ++z) s += part[(size_t)z * count + i];
        out[i] = s;
    }
}

// part[z][n] = sum of X[m][n] over the rows m of slice z: the slice's rows
// split into kColGroups consecutive groups, each summed in row order by one
// thread of a 32-column block, then the groups added in group order.
constexpr int kColGroups = 8;
__global__ void __launch_bounds__(32 * kColGroups) k_colsum_slices(const float* __restrict__ X, int64_t M, int N,
                                                                   int64_t rows_per, float* __restrict__ part) {
    __shared__ float acc[kColGroups][32];
    const int n = blockIdx.x * 32 + threadIdx.x;
    const int64_t m0 = (int64_t)blockIdx.y * rows_per, m1 = min(M, m0 + rows_per);
    const int64_t per = (rows_per + kColGroups - 1) / kColGroups;
    const int64_t a = m0 + threadIdx.y * per, b = min(m1, a + per);
    float s = 0.0f;
    if (n < N) {
#pragma unroll 8
        for (int64_t m = a; m < b; ++m) s += X[m * N + n];
    }
    acc[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && n < N) {
        float t = 0.0f;
#pragma unroll
        for (int y = 0; y < kColGroups; ++y) t += acc[y][threadIdx.x];
        part[(size_t)blockIdx.y * N + n] = t;
    }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
    }
}

unsigned grid_of(int64_t n, int threads, int64_t cap = 152 * 16) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min(b, cap));
}

// Offsets of the parameter blocks.
struct Layout {
    int64_t W1, b1, W2, b2, n;
    explicit Layout(const MlpState& s) {
        W1 = 0;
        b1 = (int64_t)s.hidden * s.P;
        W2 = b1 + s.hidden;
        b2 = W2 + (int64_t)s.dim * s.hidden;
        n = b2 + s.dim;
    }
};

int slices_for(int64_t B) { return (int)std::max<int64_t>(1, std::min<int64_t>(32, (B + 127) / 128)); }

cudaError_t ensure_weight_tiles(MlpState& s) {
    const size_t need = tile_b_elems(s.hidden, s.P) + tile_b_elems(s.dim, s.hidden) + tile_b_elems(s.hidden, s.dim);
    if (s.wt && s.wt_elems >= need) return cudaSuccess;
    if (s.wt) cudaFree(s.wt);
    s.wt = nullptr;
    s.wt_elems = 0;
    cudaError_t e = cudaMalloc(&s.wt, sizeof(float) * need);
    if (e == cudaSuccess) s.wt_elems = need;
    return e;
}

// Both forward products on mlp_fwd.cu's kernel (BF16 activations, layer
// shapes it takes).
bool fwd_fast(const MlpState& s) {
    return s.act == LINE_DTYPE_BF16 && fwd_tc_supported(s.hidden, s.P) && fwd_tc_supported(s.dim, s.hidden);
}

cudaError_t ensure_w16(MlpState& s) {
    // W1, W2 and W2^T as hi/lo tiles
    const size_t need = fwd_w16_elems(s.hidden, s.P) + 2 * fwd_w16_elems(s.dim, s.hidden);
    if (s.w16 && s.w16_elems >= need) return cudaSuccess;
    if (s.w16) cudaFree(s.w16);
    s.w16 = nullptr;
    s.w16_elems = 0;
    cudaError_t e = cudaMalloc(&s.w16, sizeof(__nv_bfloat16) * need);
    if (e == cudaSuccess) s.w16_elems = need;
    return e;
}

cudaError_t ensure_cap(MlpState& s, int64_t rows) {
    if (rows <= s.cap) return cudaSuccess;
    const int64_t cap = std::max<int64_t>(rows, 1024);
    if (s.arena) cudaFree(s.arena);
    s.arena = nullptr;
    s.rows = nullptr;
    s.Xb = s.Hb = s.sum_tmp = nullptr;
    s.Tb = s.A1 = s.Yb = s.dH = s.part = nullptr;
    s.rowloss = nullptr;
    s.gY = s.gA = nullptr;
    s.cap = 0;
    const size_t act = s.act == LINE_DTYPE_F32 ? 4 : 2;
    const int S = std::max(32, kWgradMaxSlices);
    s.part_elems = (size_t)S * std::max<int64_t>((int64_t)s.hidden * s.P, (int64_t)s.dim * s.hidden);
    // every batch buffer in one allocation, each at a 256-byte boundary
    const bool hilo = s.act == LINE_DTYPE_BF16;
    const size_t sizes[] = {sizeof(int32_t) * cap,
                            act * cap * s.P,
                            sizeof(float) * cap * s.dim,
                            sizeof(float) * cap * s.hidden,
                            act * cap * s.hidden,
                            sizeof(float) * cap * s.dim,
                            sizeof(float) * cap * s.hidden,
                            sizeof(float) * s.part_elems,
                            sizeof(double) * cap,
                            fixed_sum_tmp_bytes(cap),
                            hilo ? sizeof(__nv_bfloat16) * 2 * cap * s.dim : 0,
                            hilo ? sizeof(__nv_bfloat16) * 2 * cap * s.hidden : 0};
    constexpr int kBufs = sizeof(sizes) / sizeof(sizes[0]);
    size_t off[kBufs], total = 0;
    for (int i = 0; i < kBufs; ++i) {
        off[i] = total;
        total += (sizes[i] + 255) / 256 * 256;
    }
    void* arena = nullptr;
    cudaError_t e = cudaMalloc(&arena, total);
    if (e != cudaSuccess) return e;
    unsigned char* b = reinterpret_cast<unsigned char*>(arena);
    s.arena = arena;
    s.rows = reinterpret_cast<int32_t*>(b + off[0]);
    s.Xb = b + off[1];
    s.Tb = reinterpret_cast<float*>(b + off[2]);
    s.A1 = reinterpret_cast<float*>(b + off[3]);
    s.Hb = b + off[4];
    s.Yb = reinterpret_cast<float*>(b + off[5]);
    s.dH = reinterpret_cast<float*>(b + off[6]);
    s.part = reinterpret_cast<float*>(b + off[7]);
    s.rowloss = reinterpret_cast<double*>(b + off[8]);
    s.sum_tmp = b + off[9];
    s.gY = hilo ? reinterpret_cast<__nv_bfloat16*>(b + off[10]) : nullptr;
    s.gA = hilo ? reinterpret_cast<__nv_bfloat16*>(b + off[11]) : nullptr;
    s.cap = cap;
    return cudaSuccess;
}

// Forward pass of rows s.rows[0..B): Xb, A1, Hb, Yb (= W2 h, before b2).
template <typename TX>
cudaError_t forward(MlpState& s, int64_t B, const Tables& t, bool targets, uint32_t* status, int64_t n_nodes,
                    cudaStream_t st) {
    const Layout L(s);
    const float* W1 = s.params + L.W1;
    const float* b1 = s.params + L.b1;
    const float* W2 = s.params + L.W2;
    TX* Xb = reinterpret_cast<TX*>(s.Xb);
    TX* Hb = reinterpret_cast<TX*>(s.Hb);
    k_mlp_gather<TX><<<grid_of(B * 32, 256), 256, 0, st>>>(s.rows, B, n_nodes, reinterpret_cast<const TX*>(s.X), s.P,
                                                            Xb, t.U, t.dtype, s.dim, targets ? s.Tb : nullptr, status);
    cudaError_t e;
    if constexpr (std::is_same<TX, __nv_bfloat16>::value) {
        if (fwd_fast(s)) {
            // H = GELU(X W1^T + b1) (and A1 = X W1^T + b1 when training),
            // then Y = H W2^T, both on the tensor cores with the weights as
            // BF16 hi/lo pairs
            if ((e = ensure_w16(s)) != cudaSuccess) return e;
            const size_t e1 = fwd_w16_elems(s.hidden, s.P);
            if ((e = fwd_tile_weights(W1, s.hidden, s.P, s.w16, st)) != cudaSuccess) return e;
            if ((e = fwd_tile_weights(W2, s.dim, s.hidden, s.w16 + e1, st)) != cudaSuccess) return e;
            if ((e = fwd_tc((int)B, s.hidden, s.P, Xb, s.w16, b1, targets ? s.A1 : nullptr, Hb, nullptr, status,
                            st)) != cudaSuccess)
                return e;
            return fwd_tc((int)B, s.dim, s.hidden, Hb, s.w16 + e1, nullptr, nullptr, nullptr, s.Yb, status, st);
        }
    }
    const bool tc = s.act == LINE_DTYPE_BF16;
    const float* W1t = nullptr;
    const float* W2t = nullptr;
    if (tc) {
        // the weights as tensor-core tiles, copied in bulk by the products
        if ((e = ensure_weight_tiles(s)) != cudaSuccess) return e;
        const size_t e1 = tile_b_elems(s.hidden, s.P);
        k_tile_b<true><<<grid_of((int64_t)e1, 256), 256, 0, st>>>(W1, s.P, s.hidden, s.P, tc_tile_n(s.hidden), s.wt);
        k_tile_b<true><<<grid_of((int64_t)tile_b_elems(s.dim, s.hidden), 256), 256, 0, st>>>(
            W2, s.hidden, s.dim, s.hidden, tc_tile_n(s.dim), s.wt + e1);
        W1t = s.wt;
        W2t = s.wt + e1;
    }
    if (tc) {
        // A1 = X W1^T + b1 and H = GELU(A1) from the product's epilogue
        const int NT = tc_tile_n(s.hidden);
        e = NT == 256 ? launch_tc<TX, float, true, true, 256, true, TX>((int)B, s.hidden, s.P, 1, Xb, s.P, W1, s.P, W1t,
                                                                       s.A1, status, st, b1, Hb)
            : NT == 128 ? launch_tc<TX, float, true, true, 128, true, TX>((int)B, s.hidden, s.P, 1, Xb, s.P, W1, s.P,
                                                                         W1t, s.A1, status, st, b1, Hb)
                        : launch_tc<TX, float, true, true, 64, true, TX>((int)B, s.hidden, s.P, 1, Xb, s.P, W1, s.P, W1t,
                                                                        s.A1, status, st, b1, Hb);
        if (e != cudaSuccess) return e;
    } else {
        if ((e = gemm<TX, float, true, true>(tc, (int)B, s.hidden, s.P, 1, Xb, s.P, W1, s.P, s.A1, status, st)) !=
            cudaSuccess)
            return e;
        k_ep_hidden<TX><<<grid_of(B * s.hidden, 256), 256, 0, st>>>(s.A1, b1, B, s.hidden, Hb);
    }
    return gemm<TX, float, true, true>(tc, (int)B, s.dim, s.hidden, 1, Hb, s.hidden, W2, s.hidden, s.Yb, status, st,
                                       W2t);
}

// Loss and gradients of the batch s.rows[0..B) into s.grads; the batch loss
// (fixed-order FP64 sum / (B D)) into *loss_dev.
template <typename TX>
cudaError_t loss_grad(MlpState& s, int64_t B, const Tables& t, uint32_t* status, int64_t n_nodes, double* loss_dev,
                      cudaStream_t st) {
    const Layout L(s);
    cudaError_t e;
    if ((e = forward<TX>(s, B, t, true, status, n_nodes, st)) != cudaSuccess) return e;
    const float* W2 = s.params + L.W2;
    const float* b2 = s.params + L.b2;
    const float scale = (float)(2.0 / ((double)B * s.dim));
    // the weight gradients on the tensor cores (BF16 activations, shapes the
    // kernel takes): dY and dA also as BF16 hi/lo pairs
    const bool tc = s.act == LINE_DTYPE_BF16;
    const bool wtc = tc && s.gY && s.gA && wgrad_tc_supported(s.dim, s.hidden) && wgrad_tc_supported(s.hidden, s.P) &&
                     B <= INT32_MAX;
    k_ep_loss<<<grid_of(B * 32, 256), 256, 0, st>>>(s.Yb, b2, s.Tb, B, s.dim, scale, s.rowloss, wtc ? s.gY : nullptr);
    // dH = dY W2, then dA = dH GELU'(a): with the tensor-core weight
    // gradients, one pass on the forward kernel (dY as its hi/lo pair, W2^T as
    // hi/lo tiles) that writes dA and its hi/lo pair
    if (wtc && fwd_fast(s) && s.w16 && dact_tc_supported(s.hidden, s.dim)) {
        __nv_bfloat16* w2t = s.w16 + fwd_w16_elems(s.hidden, s.P) + fwd_w16_elems(s.dim, s.hidden);
        if ((e = fwd_tile_weights_t(W2, s.hidden, s.dim, w2t, st)) != cudaSuccess) return e;
        if ((e = dact_tc((int)B, s.hidden, s.dim, s.gY, s.gY + B * s.dim, w2t, s.A1, s.dH, s.gA, status, st)) !=
            cudaSuccess)
            return e;
    } else {
        const float* W2tT = nullptr;
        if (tc) {
            if ((e = ensure_weight_tiles(s)) != cudaSuccess) return e;
            float* dst = s.wt + tile_b_elems(s.hidden, s.P) + tile_b_elems(s.dim, s.hidden);
            k_tile_b<false><<<grid_of((int64_t)tile_b_elems(s.hidden, s.dim), 256), 256, 0, st>>>(
                W2, s.hidden, s.hidden, s.dim, tc_tile_n(s.hidden), dst);
            W2tT = dst;
        }
        if ((e = gemm<float, float, true, false>(tc, (int)B, s.hidden, s.dim, 1, s.Yb, s.dim, W2, s.hidden, s.dH,
                                                 status, st, W2tT)) != cudaSuccess)
            return e;
        k_ep_dact<<<grid_of(B * s.hidden, 256), 256, 0, st>>>(s.dH, s.A1, B * s.hidden, wtc ? s.gA : nullptr);
    }
    const TX* Xb = reinterpret_cast<const TX*>(s.Xb);
    const TX* Hb = reinterpret_cast<const TX*>(s.Hb);
    const int S = slices_for(B);
    if constexpr (std::is_same<TX, __nv_bfloat16>::value) {
        if (wtc) {
            // gW2 = dY^T H and gW1 = dA^T X, split over the batch, the slices
            // summed in order
            const int SW = wgrad_slices((int)B);
            const int64_t nW2 = (int64_t)s.dim * s.hidden, nW1 = (int64_t)s.hidden * s.P;
            if ((e = wgrad_tc(s.dim, s.hidden, (int)B, s.gY, s.gY + B * s.dim, Hb, s.part, status, st)) != cudaSuccess)
                return e;
            k_sum_slices<<<grid_of(nW2, 256), 256, 0, st>>>(s.part, SW, nW2, s.grads + L.W2);
            if ((e = wgrad_tc(s.hidden, s.P, (int)B, s.gA, s.gA + B * s.hidden, Xb, s.part, status, st)) !=
                cudaSuccess)
                return e;
            k_sum_slices<<<grid_of(nW1, 256), 256, 0, st>>>(s.part, SW, nW1, s.grads + L.W1);
        }
    }
    if (!wtc) {
        // gW2 = dY^T H
        if ((e = gemm<float, TX, false, false>(tc, s.dim, s.hidden, (int)B, S, s.Yb, s.dim, Hb, s.hidden, s.part,
                                               status, st)) != cudaSuccess)
            return e;
        k_sum_slices<<<grid_of((int64_t)s.dim * s.hidden, 256), 256, 0, st>>>(s.part, S, (int64_t)s.dim * s.hidden,
                                                                              s.grads + L.W2);
        // gW1 = dA^T X
        if ((e = gemm<float, TX, false, false>(tc, s.hidden, s.P, (int)B, S, s.dH, s.hidden, Xb, s.P, s.part,
                                               status, st)) != cudaSuccess)
            return e;
        k_sum_slices<<<grid_of((int64_t)s.hidden * s.P, 256), 256, 0, st>>>(s.part, S, (int64_t)s.hidden * s.P,
                                                                           s.grads + L.W1);
    }
    // bias gradients: column sums in slices of rows, slices summed in order
    const int64_t rows_per = (B + S - 1) / S;
    k_colsum_slices<<<dim3((s.hidden + 31) / 32, S), dim3(32, kColGroups), 0, st>>>(s.dH, B, s.hidden, rows_per, s.part);
    k_sum_slices<<<grid_of(s.hidden, 256), 256, 0, st>>>(s.part, S, s.hidden, s.grads + L.b1);
    k_colsum_slices<<<dim3((s.dim + 31) / 32, S), dim3(32, kColGroups), 0, st>>>(s.Yb, B, s.dim, rows_per, s.part);
    k_sum_slices<<<grid_of(s.dim, 256), 256, 0, st>>>(s.part, S, s.dim, s.grads + L.b2);
    if ((e = fixed_sum_f64(s.rowloss, B, reinterpret_cast<double*>(s.sum_tmp), loss_dev, st)) != cudaSuccess) return e;
    return cudaGetLastError();
}

__global__ void k_scale_loss(double* loss, double inv) { *loss *= inv; }

}  // namespace

}  // namespace line

using namespace line;

namespace {

line_status mlp_ready(line_ctx* c, const char* what, bool need_features) {
    if (!c->mlp) return fail(c, LINE_ERR_STATE, "%s: no MLP (call line_mlp_create)", what);
    if (!c->tab[c->mlp->order].ready || c->tab[c->mlp->order].dim != c->mlp->dim)
        return fail(c, LINE_ERR_STATE, "%s: the tables of order %d (dim %d) are gone", what, c->mlp->order,
                    c->mlp->dim);
    if (need_features && !c->mlp->has_features)
        return fail(c, LINE_ERR_STATE, "%s: no inputs (call line_mlp_features or line_mlp_features_rows)", what);
    return LINE_OK;
}

// Device copy of a node list (host or device buffer), into s.nodes.
cudaError_t upload_nodes(MlpState& s, const int32_t* nodes, int64_t n, cudaStream_t st) {
    if (n > s.nodes_cap) {
        if (s.nodes) cudaFree(s.nodes);
        s.nodes = nullptr;
        s.nodes_cap = 0;
        cudaError_t e = cudaMalloc(&s.nodes, sizeof(int32_t) * n);
        if (e != cudaSuccess) return e;
        s.nodes_cap = n;
    }
    return cudaMemcpyAsync(s.nodes, nodes, sizeof(int32_t) * n, cudaMemcpyDefault, st);
}

}  // namespace

extern "C" {

line_status line_mlp_create(line_ctx* c, int order, int hidden, int act_dtype, uint64_t seed) {
    NvtxRange nvtx("line_mlp_create");
    line_status st = enter(c);
    if (st) return st;
    if (!c->has_graph) return fail(c, LINE_ERR_STATE, "line_mlp_create: no graph");
    if ((order != 1 && order != 2) || hidden < 1 || hidden > 4096 ||
        (act_dtype != LINE_DTYPE_F32 && act_dtype != LINE_DTYPE_BF16))
        return fail(c, LINE_ERR_ARG, "line_mlp_create: bad order, hidden width or activation type");
    const Tables& t = c->tab[order];
    if (!t.ready) return fail(c, LINE_ERR_STATE, "line_mlp_create: no tables of order %d", order);
    MlpState* s = c->mlp;
    c->mlp = nullptr;
    cudaError_t e = cudaSuccess;
    if (s && s->order == order && s->dim == t.dim && s->hidden == hidden && s->act == act_dtype &&
        s->n_nodes == c->n_nodes) {
        // an MLP of the same shape: its allocations are kept, its contents
        // start over below (weights, optimiser state, inputs)
        s->t = 0;
        s->has_features = false;
    } else {
        mlp_destroy(s);
        s = new MlpState();
        s->order = order;
        s->dim = t.dim;
        s->hidden = hidden;
        s->P = (t.dim + 1 + 15) / 16 * 16;
        s->act = act_dtype;
        s->n_nodes = c->n_nodes;
        const Layout L0(*s);
        s->n_params = L0.n;
        // params, grads, m and v in one allocation, each at a 256-byte boundary
        const size_t pbs = (sizeof(float) * L0.n + 255) / 256 * 256;
        e = cudaMalloc(&s->params, 4 * pbs);
        if (e == cudaSuccess) {
            unsigned char* b = reinterpret_cast<unsigned char*>(s->params);
            s->grads = reinterpret_cast<float*>(b + pbs);
            s->m = reinterpret_cast<float*>(b + 2 * pbs);
            s->v = reinterpret_cast<float*>(b + 3 * pbs);
        }
        if (e == cudaSuccess) e = cudaMalloc(&s->X, (size_t)c->n_nodes * s->P * elem_size(act_dtype));
    }
    const Layout L(*s);
    const size_t pb = sizeof(float) * L.n;
    // inputs not yet computed are zero (line_mlp_features_rows may compute a subset)
    if (e == cudaSuccess) e = cudaMemsetAsync(s->X, 0, (size_t)c->n_nodes * s->P * elem_size(act_dtype), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->m, 0, pb, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->v, 0, pb, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->grads, 0, pb, c->stream);
    if (e == cudaSuccess) {
        const float s1 = (float)(1.0 / sqrt((double)(t.dim + 1)));
        const float s2 = (float)(1.0 / sqrt((double)hidden));
        k_mlp_init<<<grid_of(L.n, 256), 256, 0, c->stream>>>(s->params, hidden, s->P, t.dim, seed, s1, s2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        mlp_destroy(s);
        return cuda_fail(c, e, "line_mlp_create");
    }
    c->mlp = s;
    return LINE_OK;
}

// Inputs of the nodes rows[0 .. n_rows) (all nodes when rows is null).
static line_status mlp_features_impl(line_ctx* c, const char* what, const uint8_t* known, const int32_t* rows,
                                     int64_t n_rows) {
    line_status st = enter(c);
    if (st) return st;
    if ((st = mlp_ready(c, what, false))) return st;
    if (!known) return fail(c, LINE_ERR_ARG, "%s: null mask", what);
    if (rows && n_rows < 0) return fail(c, LINE_ERR_ARG, "%s: bad row count", what);
    MlpState& s = *c->mlp;
    if (rows && n_rows == 0) return LINE_OK;
    const Tables& t = c->tab[s.order];
    if ((st = ensure_row_ptr(c))) return st;
    // scratch kept in the MLP state (grown, never shrunk)
    const int64_t max_hubs = HubScratch(c->n_nodes, c->n_arcs).max_hubs;
    cudaError_t e = cudaSuccess;
    if (!s.kmask) e = cudaMalloc(&s.kmask, (size_t)c->n_nodes);
    if (e == cudaSuccess && !s.flag) e = cudaMalloc(&s.flag, sizeof(uint32_t));
    const HubScratch hs(c->n_nodes, c->n_arcs);
    const size_t hub_bytes = hs.bytes(s.dim);
    if (e == cudaSuccess && s.hubs_cap < (int64_t)hub_bytes) {
        if (s.hubs) cudaFree(s.hubs);
        s.hubs = nullptr;
        s.hubs_cap = 0;
        if ((e = cudaMalloc(&s.hubs, hub_bytes)) == cudaSuccess) s.hubs_cap = (int64_t)hub_bytes;
    }
    if (e == cudaSuccess && rows && s.frows_cap < n_rows) {
        if (s.frows) cudaFree(s.frows);
        s.frows = nullptr;
        s.frows_cap = 0;
        if ((e = cudaMalloc(&s.frows, sizeof(int32_t) * (size_t)n_rows)) == cudaSuccess) s.frows_cap = n_rows;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    cudaStream_t str = c->stream;
    // hub scratch: the listed-hub bitmap, [count] then the listed hub
    // nodes, the chunk offsets (off, poff), the chunk-sum counts and the
    // chunk sums (256-byte aligned)
    uint32_t* hub_map = s.hubs;
    uint32_t* hubs = hub_map + hs.map_words;
    uint32_t* hub_off = hubs + hs.list_words();
    uint32_t* hub_poff = hub_off + hs.off_words();
    uint32_t* hub_pcnt = hub_poff + hs.off_words();
    float* hub_part = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(hub_pcnt + hs.max_multi) + 255) & ~(uintptr_t)255);
    int32_t* rd = rows ? s.frows : nullptr;
    e = cudaMemcpyAsync(s.kmask, known, c->n_nodes, cudaMemcpyDefault, str);
    if (e == cudaSuccess && rows) e = cudaMemcpyAsync(rd, rows, sizeof(int32_t) * n_rows, cudaMemcpyDefault, str);
    if (e == cudaSuccess) e = cudaMemsetAsync(hub_map, 0, sizeof(uint32_t) * ((size_t)hs.map_words + 1), str);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.flag, 0, sizeof(uint32_t), str);
    if (e == cudaSuccess) {
        // ids out of range are refused before any work: the flag stops the
        // input kernels
        if (rows) k_check_rows<<<grid_of(n_rows, 256, 152 * 16), 256, 0, str>>>(rd, n_rows, c->n_nodes, s.flag);
        const int64_t count = rows ? n_rows : c->n_nodes;
        FeatParams fp{c->n_nodes, c->row_ptr, c->dst,  c->deg,   t.U,      s.kmask, s.P,    s.X,   hub_map, hubs + 1,
                      hubs,       hub_off,    hub_poff, hub_part, hub_pcnt, rd,      n_rows, s.flag};
        if (s.act == LINE_DTYPE_F32)
            e = t.dtype == LINE_DTYPE_F32 ? features_for<LINE_DTYPE_F32, float>(s.dim, fp, count, max_hubs, str)
                                          : features_for<LINE_DTYPE_BF16, float>(s.dim, fp, count, max_hubs, str);
        else
            e = t.dtype == LINE_DTYPE_F32 ? features_for<LINE_DTYPE_F32, __nv_bfloat16>(s.dim, fp, count, max_hubs, str)
                                          : features_for<LINE_DTYPE_BF16, __nv_bfloat16>(s.dim, fp, count, max_hubs, str);
    }
    uint32_t bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, s.flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, str);
    if (e == cudaSuccess) e = cudaStreamSynchronize(str);
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    if (bad) return fail(c, LINE_ERR_ARG, "%s: a row id is out of range", what);
    s.has_features = true;
    return LINE_OK;
}

line_status line_mlp_features(line_ctx* c, const uint8_t* known) {
    NvtxRange nvtx("line_mlp_features");
    return mlp_features_impl(c, "line_mlp_features", known, nullptr, 0);
}

line_status line_mlp_features_rows(line_ctx* c, const uint8_t* known, const int32_t* rows, int64_t n_rows) {
    NvtxRange nvtx("line_mlp_features_rows");
    if (!rows) return c ? fail(c, LINE_ERR_ARG, "line_mlp_features_rows: null rows") : LINE_ERR_ARG;
    return mlp_features_impl(c, "line_mlp_features_rows", known, rows, n_rows);
}

line_status line_mlp_get_features(line_ctx* c, float* out) {
    line_status st = enter(c);
    if (st) return st;
    if ((st = mlp_ready(c, "line_mlp_get_features", true))) return st;
    if (!out) return fail(c, LINE_ERR_ARG, "line_mlp_get_features: null output");
    MlpState& s = *c->mlp;
    const size_t n = (size_t)c->n_nodes * s.P;
    if (s.act == LINE_DTYPE_F32) {
        CK(cudaMemcpyAsync(out, s.X, n * 4, cudaMemcpyDefault, c->stream), "line_mlp_get_features");
        CK(cudaStreamSynchronize(c->stream), "line_mlp_get_features");
        return LINE_OK;
    }
    void* buf = nullptr;
    CK(cudaMalloc(&buf, n * 4), "line_mlp_get_features");
    cudaError_t e = convert_rows(s.X, LINE_DTYPE_BF16, buf, LINE_DTYPE_F32, nullptr, c->n_nodes, s.P, c->n_nodes,
                                 c->status, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, buf, n * 4, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(c, e, "line_mlp_get_features");
    return LINE_OK;
}

line_status line_mlp_get_params(line_ctx* c, float* out, int64_t* n_params) {
    line_status st = enter(c);
    if (st) return st;
    if (!c->mlp) return fail(c, LINE_ERR_STATE, "line_mlp_get_params: no MLP");
    if (n_params) *n_params = c->mlp->n_params;
    if (out) {
        CK(cudaMemcpyAsync(out, c->mlp->params, sizeof(float) * c->mlp->n_params, cudaMemcpyDefault, c->stream),
           "line_mlp_get_params");
        CK(cudaStreamSynchronize(c->stream), "line_mlp_get_params");
    }
    return LINE_OK;
}

line_status line_mlp_set_params(line_ctx* c, const float* in) {
    line_status st = enter(c);
    if (st) return st;
    if (!c->mlp) return fail(c, LINE_ERR_STATE, "line_mlp_set_params: no MLP");
    if (!in) return fail(c, LINE_ERR_ARG, "line_mlp_set_params: null input");
    MlpState& s = *c->mlp;
    const size_t pb = sizeof(float) * s.n_params;
    CK(cudaMemcpyAsync(s.params, in, pb, cudaMemcpyDefault, c->stream), "line_mlp_set_params");
    // a new starting point: the optimiser state restarts
    CK(cudaMemsetAsync(s.m, 0, pb, c->stream), "line_mlp_set_params");
    CK(cudaMemsetAsync(s.v, 0, pb, c->stream), "line_mlp_set_params");
    CK(cudaStreamSynchronize(c->stream), "line_mlp_set_params");
    s.t = 0;
    return LINE_OK;
}

line_status line_mlp_grad(line_ctx* c, const int32_t* rows, int64_t n_rows, float* grads_out, double* loss_out) {
    NvtxRange nvtx("line_mlp_grad");
    line_status st = enter(c);
    if (st) return st;
    if ((st = mlp_ready(c, "line_mlp_grad", true))) return st;
    if (!rows || n_rows < 1 || n_rows > kMlpMaxBatch)
        return fail(c, LINE_ERR_ARG, "line_mlp_grad: n_rows must be 1..%lld", (long long)kMlpMaxBatch);
    MlpState& s = *c->mlp;
    const Tables& t = c->tab[s.order];
    CK(ensure_cap(s, n_rows), "line_mlp_grad");
    CK(cudaMemcpyAsync(s.rows, rows, sizeof(int32_t) * n_rows, cudaMemcpyDefault, c->stream), "line_mlp_grad");
    cudaError_t e = s.act == LINE_DTYPE_F32
                        ? loss_grad<float>(s, n_rows, t, c->status, c->n_nodes, c->dscratch, c->stream)
                        : loss_grad<__nv_bfloat16>(s, n_rows, t, c->status, c->n_nodes, c->dscratch, c->stream);
    if (e == cudaSuccess) {
        k_scale_loss<<<1, 1, 0, c->stream>>>(c->dscratch, 1.0 / ((double)n_rows * s.dim));
        e = cudaGetLastError();
    }
    double loss = 0.0;
    if (e == cudaSuccess && grads_out)
        e = cudaMemcpyAsync(grads_out, s.grads, sizeof(float) * s.n_params, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&loss, c->dscratch, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "line_mlp_grad");
    if ((st = check_status(c, "line_mlp_grad"))) return st;
    if (loss_out) *loss_out = loss;
    return LINE_OK;
}

line_status line_mlp_train(line_ctx* c, const int32_t* nodes, int64_t n_nodes, int64_t steps, int64_t batch,
                           double lr, uint64_t seed, uint64_t step_offset, double* losses_out) {
    NvtxRange nvtx("line_mlp_train");
    line_status st = enter(c);
    if (st) return st;
    if ((st = mlp_ready(c, "line_mlp_train", true))) return st;
    if (!nodes || n_nodes < 1 || steps < 0 || batch < 1 || batch > kMlpMaxBatch || !(lr >= 0.0))
        return fail(c, LINE_ERR_ARG, "line_mlp_train: bad arguments");
    if (steps == 0) return LINE_OK;
    MlpState& s = *c->mlp;
    const Tables& t = c->tab[s.order];
    cudaStream_t str = c->stream;
    CK(ensure_cap(s, batch), "line_mlp_train");
    CK(upload_nodes(s, nodes, n_nodes, str), "line_mlp_train");
    if (steps > s.loss_cap) {
        if (s.losses) cudaFree(s.losses);
        s.losses = nullptr;
        s.loss_cap = 0;
        CK(cudaMalloc(&s.losses, sizeof(double) * steps), "line_mlp_train");
        s.loss_cap = steps;
    }
    // node ids out of range are reported by the gather (status word)
    for (int64_t k = 0; k < steps; ++k) {
        const uint64_t gstep = step_offset + (uint64_t)k;
        k_mlp_batch<<<grid_of(batch, 256), 256, 0, str>>>(s.nodes, n_nodes, seed, gstep * (uint64_t)batch, batch,
                                                          s.rows);
        cudaError_t e = s.act == LINE_DTYPE_F32
                            ? loss_grad<float>(s, batch, t, c->status, c->n_nodes, s.losses + k, str)
                            : loss_grad<__nv_bfloat16>(s, batch, t, c->status, c->n_nodes, s.losses + k, str);
        if (e != cudaSuccess) return cuda_fail(c, e, "line_mlp_train");
        ++s.t;
        const float c1 = (float)(1.0 / (1.0 - pow(0.9, (double)s.t)));
        const float c2 = (float)(1.0 / (1.0 - pow(0.999, (double)s.t)));
        k_adam<<<grid_of(s.n_params, 256), 256, 0, str>>>(s.params, s.grads, s.m, s.v, s.n_params, (float)lr, c1, c2);
        CK(cudaGetLastError(), "line_mlp_train");
    }
    if (losses_out) {
        std::vector<double> tmp(steps);
        CK(cudaMemcpyAsync(tmp.data(), s.losses, sizeof(double) * steps, cudaMemcpyDeviceToHost, str), "line_mlp_train");
        CK(cudaStreamSynchronize(str), "line_mlp_train");
        const double inv = 1.0 / ((double)batch * s.dim);
        for (int64_t k = 0; k < steps; ++k) losses_out[k] = tmp[k] * inv;
    }
    return check_status(c, "line_mlp_train");
}

line_status line_mlp_predict(line_ctx* c, const int32_t* rows, int64_t n_rows, float* y_out) {
    NvtxRange nvtx("line_mlp_predict");
    line_status st = enter(c);
    if (st) return st;
    if ((st = mlp_ready(c, "line_mlp_predict", true))) return st;
    if (!rows || n_rows < 0) return fail(c, LINE_ERR_ARG, "line_mlp_predict: bad arguments");
    if (n_rows == 0) return LINE_OK;
    MlpState& s = *c->mlp;
    const Tables& t = c->tab[s.order];
    cudaStream_t str = c->stream;
    const int64_t chunk = std::min<int64_t>(n_rows, kMlpMaxBatch);
    CK(ensure_cap(s, chunk), "line_mlp_predict");
    float* ybuf = nullptr;
    if (y_out) CK(cudaMalloc(&ybuf, sizeof(float) * n_rows * s.dim), "line_mlp_predict");
    const Layout L(s);
    cudaError_t e = cudaSuccess;
    // all requested ids in one copy; each chunk then takes its slice on the device
    if (s.frows_cap < n_rows) {
        if (s.frows) cudaFree(s.frows);
        s.frows = nullptr;
        s.frows_cap = 0;
        if ((e = cudaMalloc(&s.frows, sizeof(int32_t) * (size_t)n_rows)) == cudaSuccess) s.frows_cap = n_rows;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.frows, rows, sizeof(int32_t) * n_rows, cudaMemcpyDefault, str);
    for (int64_t r0 = 0; r0 < n_rows && e == cudaSuccess; r0 += chunk) {
        const int64_t B = std::min(chunk, n_rows - r0);
        e = cudaMemcpyAsync(s.rows, s.frows + r0, sizeof(int32_t) * B, cudaMemcpyDeviceToDevice, str);
        if (e == cudaSuccess)
            e = s.act == LINE_DTYPE_F32 ? forward<float>(s, B, t, false, c->status, c->n_nodes, str)
                                        : forward<__nv_bfloat16>(s, B, t, false, c->status, c->n_nodes, str);
        if (e == cudaSuccess) {
            if (ybuf)
                k_ep_predict<<<grid_of(B * s.dim, 256), 256, 0, str>>>(s.Yb, s.params + L.b2, B, s.dim, nullptr, 0,
                                                                       ybuf + r0 * s.dim, LINE_DTYPE_F32);
            else
                k_ep_predict<<<grid_of(B * s.dim, 256), 256, 0, str>>>(s.Yb, s.params + L.b2, B, s.dim, s.rows,
                                                                       c->n_nodes, t.U, t.dtype);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && ybuf) e = cudaMemcpyAsync(y_out, ybuf, sizeof(float) * n_rows * s.dim, cudaMemcpyDefault, str);
    if (e == cudaSuccess) e = cudaStreamSynchronize(str);
    if (ybuf) cudaFree(ybuf);
    if (e != cudaSuccess) return cuda_fail(c, e, "line_mlp_predict");
    return check_status(c, "line_mlp_predict");
}

}  // extern "C"
