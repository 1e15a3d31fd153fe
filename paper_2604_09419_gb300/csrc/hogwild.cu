// Hogwild schedule (LINE_MODE_HOGWILD): the local path of Algorithm 1, with
// LineUpdate applied pair after pair and at once.  Many workers run it
// concurrently on the shared tables without locks, in the manner of Hogwild
// (Recht et al., NeurIPS 2011).  There is no grouping pass, no delta slab
// and no apply kernel.
//
// A worker is a lane group (the row geometry of the minibatch kernels: L
// lanes per row, E values per lane).  Worker w takes samples w, w + n_w,
// w + 2 n_w, ... of the chunk's records (written by the pre-pass) and, per
// sample:
//   - loads each distinct row of the sample once (the U row of u and the
//     context rows of v, n_1 .. n_K; in order 1 the context table is U, so
//     u may also be a context row) into its shared-memory stage;
//   - runs the K+1 calls in order on the staged rows: x = U[u], c = Ctx[y],
//     s = x . c, g = eta (1 - sigma(s)) or -eta alpha_neg sigma(s),
//     U[u] <- x + (g c - eta lambda x), Ctx[y] <- c + (g x - eta lambda c)
//     (both from the values before the call; Ctx[y] written last);
//   - adds each call's change of the context row to the table at once, and
//     the U row's net change (final - loaded) after the last call, with
//     atomic adds: FP32 rows by vector float adds, BF16 rows by BF16 adds
//     of the change plus one unit in the last place of uniform noise, which
//     makes the rounding stochastic in expectation.
// Inside a sample this is exactly the sequential order of the calls.  Across
// workers, reads are not synchronised, so a sample may compute on rows that
// other workers are changing, but no worker's change is overwritten by
// another's, as in CPU Hogwild where every element update is an in-place
// add.  Overwriting whole rows instead loses almost every update of the hub
// rows once thousands of workers run.  With one worker the run is the
// sequential per-pair SGD.  eta is the schedule's value at the first sample
// of the sample's batch.
#include <algorithm>
#include <mutex>
#include <vector>

#include "line_internal.cuh"
#include "rows.cuh"

namespace line {
namespace {

constexpr int kHogWarps = 4;   // warps per block, at most (fewer when a block's stages exceed the shared memory)

// Shared memory per lane group: the staged rows, then the record and the
// first-occurrence slot of each slot, rounded up to 16 bytes.
__host__ __device__ inline size_t group_bytes(int dim, int K) {
    return (sizeof(float) * (size_t)(K + 2) * dim + sizeof(int32_t) * 2 * (K + 2) + 15) & ~(size_t)15;
}

// Spacing of BF16 values (8 significant bits) around v; below the normal
// range, that of the smallest normal binade.
__device__ __forceinline__ float bf16_ulp(float v) {
    const uint32_t e = (__float_as_uint(v) >> 23) & 0xFFu;
    return __uint_as_float((e > 8u ? e - 7u : 1u) << 23);
}

// table[row] += d for this lane's values, as fire-and-forget atomics.
// FP32: vector float adds.  BF16: the hardware BF16 add rounds to nearest,
// which would drop every change below half a unit in the last place; so
// each change first gets uniform noise of one unit in the last place of
// `ref` (the value the worker saw; noise from the SplitMix64 bits of the
// row write's key, with `key` in place of the batch start).  The rounded
// sum is then correct in expectation, as with stochastic rounding.
template <int D, int DT>
__device__ __forceinline__ void add_row(void* table, int64_t row, int lig, const float (&d)[Geom<D, DT>::E],
                                        const float (&ref)[Geom<D, DT>::E], uint64_t seed, uint64_t key,
                                        uint32_t table_id) {
    using G = Geom<D, DT>;
    if constexpr (DT == LINE_DTYPE_F32) {
        float4* p = reinterpret_cast<float4*>(reinterpret_cast<float*>(table) + row * D + lig * G::E);
#pragma unroll
        for (int q = 0; q < G::NV; ++q) atomicAdd(p + q, make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]));
    } else {
        __nv_bfloat162* p = reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(table) + row * D + lig * G::E);
#pragma unroll
        for (int q = 0; q < G::NV; ++q) {
            const uint32_t k4 = (uint32_t)((lig * G::E + 4 * q) >> 2);
            const uint64_t r = sr_bits(seed, table_id, (uint64_t)row, key, k4);
            float dd[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float u = (float)((uint32_t)(r >> (16 * i)) & 0xFFFFu) * (1.0f / 65536.0f) - 0.5f;
                dd[i] = fmaf(u, bf16_ulp(ref[4 * q + i]), d[4 * q + i]);
            }
            const __nv_bfloat162 lo = __floats2bfloat162_rn(dd[0], dd[1]), hi = __floats2bfloat162_rn(dd[2], dd[3]);
            // one 8-byte vector reduction (two BF16 pairs)
            asm volatile("red.global.add.noftz.v2.bf16x2 [%0], {%1, %2};" ::"l"(p + 2 * q),
                         "r"(*reinterpret_cast<const uint32_t*>(&lo)), "r"(*reinterpret_cast<const uint32_t*>(&hi))
                         : "memory");
        }
    }
}

template <int D, int DT>
__global__ void __launch_bounds__(kHogWarps * 32) k_hogwild(HogwildParams p) {
    using G = Geom<D, DT>;
    extern __shared__ __align__(16) unsigned char s_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G::L, lig = lane % G::L;
    const int R = p.K + 2;
    const uint32_t gm = group_mask<G::L>(grp);
    const int gid = warp * G::GPW + grp;
    unsigned char* base = s_raw + (size_t)gid * group_bytes(D, p.K);
    float* stage = reinterpret_cast<float*>(base);
    int32_t* srow = reinterpret_cast<int32_t*>(stage + (size_t)R * D);
    int32_t* sid = srow + R;
    const int64_t worker = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * G::GPW + grp;
    const int64_t nw = p.workers;
    const int64_t n = p.chunk_samples;
    // every lane of the warp runs the same number of rounds (the dot
    // products reduce over full-warp shuffles)
    const int64_t rounds = (n + nw - 1) / nw;
    const uint32_t ctx_tab = p.order == 2 ? 1u : 0u;
    void* ctx = p.order == 2 ? p.C : p.U;
    for (int64_t r = 0; r < rounds; ++r) {
        const int64_t s = r * nw + worker;
        const bool active = worker < nw && s < n;
        if (R <= G::L) {
            // one slot per lane: the first slot of the worker holding the
            // same row of the same table, by matching keys across the warp
            int32_t row = 0;
            if (active && lig < R) {
                row = __ldg(p.rec + s * R + lig);
                if (row < 0 || row >= p.n_nodes) {
                    atomicOr(p.status, DEV_ERR_INDEX);
                    row = 0;
                }
            }
            const uint32_t tk = lig == 0 ? 0u : ctx_tab;
            const unsigned long long key = lig < R ? ((unsigned long long)gid << 40) | ((unsigned long long)tk << 32) |
                                                         (unsigned long long)(uint32_t)row
                                                   : (1ull << 63) | (unsigned long long)lane;
            const unsigned m = __match_any_sync(0xFFFFFFFFu, key);
            if (lig < R) {
                srow[lig] = row;
                sid[lig] = __ffs(m) - 1 - grp * G::L;
            }
        } else {
            for (int k = lig; k < R; k += G::L) {
                int32_t row = active ? __ldg(p.rec + s * R + k) : 0;
                if (active && (row < 0 || row >= p.n_nodes)) {
                    atomicOr(p.status, DEV_ERR_INDEX);
                    row = 0;
                }
                srow[k] = row;
            }
            __syncwarp(gm);
            for (int k = lig; k < R; k += G::L) {
                const uint32_t tk = k == 0 ? 0u : ctx_tab;
                int id = k;
                for (int q = 0; q < k; ++q) {
                    const uint32_t tq = q == 0 ? 0u : ctx_tab;
                    if (tq == tk && srow[q] == srow[k]) {
                        id = q;
                        break;
                    }
                }
                sid[k] = id;
            }
        }
        __syncwarp(gm);
        // the U row into registers, the distinct context rows into the
        // stage, up to CH loads in flight per lane
        constexpr int CH = 4;
        float x[G::E], x0[G::E];
        if (active) {
            for (int k0 = 0; k0 < R; k0 += CH) {
                float v[CH][G::E];
#pragma unroll
                for (int kk = 0; kk < CH; ++kk) {
                    const int k = k0 + kk;
                    if (k < R && sid[k] == k) load_row<D, DT>(k == 0 ? p.U : ctx, srow[k], lig, v[kk]);
                }
                if (k0 == 0) {
#pragma unroll
                    for (int e = 0; e < G::E; ++e) x0[e] = v[0][e];
                }
#pragma unroll
                for (int kk = 0; kk < CH; ++kk) {
                    const int k = k0 + kk;
                    if (k > 0 && k < R && sid[k] == k) {
                        float4* st = reinterpret_cast<float4*>(stage + (size_t)k * D + lig * G::E);
#pragma unroll
                        for (int q = 0; q < G::NV; ++q)
                            st[q] = make_float4(v[kk][4 * q], v[kk][4 * q + 1], v[kk][4 * q + 2], v[kk][4 * q + 3]);
                    }
                }
            }
        } else {
#pragma unroll
            for (int e = 0; e < G::E; ++e) x0[e] = 0.0f;
        }
#pragma unroll
        for (int e = 0; e < G::E; ++e) x[e] = x0[e];
        __syncwarp(gm);
        const uint32_t sl = active ? (uint32_t)s : 0u;  // s < 2^26 within a chunk
        const uint64_t t = p.t_chunk + sl;
        float eta = p.lr0;
        if (p.lr_schedule == 1) {
            const uint64_t t0 = p.t_chunk + (uint64_t)(sl / (uint32_t)p.batch) * (uint64_t)p.batch;
            float f = t0 >= p.lr_total ? 0.0f : (float)(p.lr_total - t0) / (float)p.lr_total;
            if (f < p.lr_floor) f = p.lr_floor;
            eta = p.lr0 * f;
        }
        const float etalam = eta * p.lambda;
        for (int j = 0; j <= p.K; ++j) {
            const int cj = sid[1 + j];
            float c[G::E];
            if (cj == 0) {
#pragma unroll
                for (int e = 0; e < G::E; ++e) c[e] = x[e];
            } else {
                const float4* ld = reinterpret_cast<const float4*>(stage + (size_t)cj * D + lig * G::E);
#pragma unroll
                for (int q = 0; q < G::NV; ++q) {
                    const float4 a = ld[q];
                    c[4 * q] = a.x;
                    c[4 * q + 1] = a.y;
                    c[4 * q + 2] = a.z;
                    c[4 * q + 3] = a.w;
                }
            }
            float sdot = 0.0f;
#pragma unroll
            for (int e = 0; e < G::E; ++e) sdot = fmaf(x[e], c[e], sdot);
            sdot = group_sum<G::L>(sdot);
            const float sig = 1.0f / (1.0f + expf(-sdot));
            const float g = j == 0 ? eta * (1.0f - sig) : -eta * p.alpha_neg * sig;
            float dc[G::E];
#pragma unroll
            for (int e = 0; e < G::E; ++e) {
                dc[e] = g * x[e] - etalam * c[e];
                x[e] = x[e] + (g * c[e] - etalam * x[e]);
            }
            if (cj == 0) {
                // order 1 with y = u: the context write comes last and stays
#pragma unroll
                for (int e = 0; e < G::E; ++e) x[e] = c[e] + dc[e];
            } else {
                float4* st = reinterpret_cast<float4*>(stage + (size_t)cj * D + lig * G::E);
#pragma unroll
                for (int q = 0; q < G::NV; ++q)
                    st[q] = make_float4(c[4 * q] + dc[4 * q], c[4 * q + 1] + dc[4 * q + 1], c[4 * q + 2] + dc[4 * q + 2],
                                        c[4 * q + 3] + dc[4 * q + 3]);
                if (active) add_row<D, DT>(ctx, srow[cj], lig, dc, c, p.seed, t * 64u + 1u + (uint64_t)j, ctx_tab);
            }
        }
        if (active) {
            float d[G::E];
#pragma unroll
            for (int e = 0; e < G::E; ++e) d[e] = x[e] - x0[e];
            add_row<D, DT>(p.U, srow[0], lig, d, x0, p.seed, t * 64u, 0u);
        }
        __syncwarp(gm);  // the stage is rewritten by the next round
    }
}

template <int D, int DT>
cudaError_t launch(const HogwildParams& p, int64_t max_workers, cudaStream_t s) {
    using G = Geom<D, DT>;
    constexpr size_t kMaxSmem = 227 * 1024;
    const size_t per_warp = (size_t)G::GPW * group_bytes(D, p.K);
    const int wpb = (int)std::min<size_t>(kHogWarps, kMaxSmem / per_warp);
    if (wpb < 1) return cudaErrorInvalidValue;  // K and D beyond one warp's shared memory (not reachable for K <= 32)
    const size_t smem = (size_t)wpb * per_warp;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    // per device: the largest stage allowed so far (the attribute only
    // grows, so every cached wave stays launchable) and the resident wave
    // for each K (the stage size depends on K)
    struct Wave {
        int dev, K, sms, per_sm;
    };
    static std::mutex mu;
    static std::vector<Wave> waves;
    static std::vector<std::pair<int, size_t>> allowed;
    std::lock_guard<std::mutex> lock(mu);
    size_t* cap = nullptr;
    for (auto& a : allowed)
        if (a.first == dev) cap = &a.second;
    if (!cap) {
        allowed.push_back({dev, 0});
        cap = &allowed.back().second;
    }
    if (*cap < smem) {
        if ((e = cudaFuncSetAttribute(k_hogwild<D, DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        *cap = smem;
    }
    int per_sm = -1, sms = 0;
    for (const Wave& w : waves)
        if (w.dev == dev && w.K == p.K) {
            per_sm = w.per_sm;
            sms = w.sms;
        }
    if (per_sm < 0) {
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hogwild<D, DT>, wpb * 32, smem)) != cudaSuccess)
            return e;
        waves.push_back({dev, p.K, sms, per_sm});
    }
    const int64_t per_block = (int64_t)wpb * G::GPW;
    const int64_t full = (int64_t)std::max(per_sm, 1) * sms * per_block;  // one resident wave
    HogwildParams q = p;
    q.workers = max_workers > 0 ? std::min<int64_t>(max_workers, full) : full;
    q.workers = std::min<int64_t>(q.workers, std::max<int64_t>(p.chunk_samples, 1));
    const unsigned grid = (unsigned)((q.workers + per_block - 1) / per_block);
    k_hogwild<D, DT><<<grid, wpb * 32, smem, s>>>(q);
    return cudaGetLastError();
}

}  // namespace

cudaError_t hogwild_chunk(const HogwildParams& p, int dim, int dtype, int64_t max_workers, cudaStream_t s) {
    const bool bf = dtype == LINE_DTYPE_BF16;
    switch (dim) {
        case 16: return bf ? launch<16, LINE_DTYPE_BF16>(p, max_workers, s) : launch<16, LINE_DTYPE_F32>(p, max_workers, s);
        case 32: return bf ? launch<32, LINE_DTYPE_BF16>(p, max_workers, s) : launch<32, LINE_DTYPE_F32>(p, max_workers, s);
        case 64: return bf ? launch<64, LINE_DTYPE_BF16>(p, max_workers, s) : launch<64, LINE_DTYPE_F32>(p, max_workers, s);
        case 128:
            return bf ? launch<128, LINE_DTYPE_BF16>(p, max_workers, s) : launch<128, LINE_DTYPE_F32>(p, max_workers, s);
        case 256:
            return bf ? launch<256, LINE_DTYPE_BF16>(p, max_workers, s) : launch<256, LINE_DTYPE_F32>(p, max_workers, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace line
