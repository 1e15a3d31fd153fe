// Minibatch-synchronous LINE training on the GPU (Algorithm 1, Eq. 2-4).
//
// A call processes its samples in chunks of whole batches.  Per chunk:
//
//   pre-pass (index work only, independent of the tables):
//     1. draws: for every sample its arc (u, v) and K negatives, kept as a
//        record (u, v, n_1..n_K), and K+2 sort items, one per row the sample
//        touches: key = (batch, row), value = (sample, slot).  Slot 0 is
//        U[u]; slots 1..K+1 are the context rows Ctx[v], Ctx[n_j] (Ctx = C
//        for second order, U for first order; C rows get ids offset by n).
//     2. a stable LSD radix sort of the items by key; equal keys keep the
//        (sample, slot) order.
//     3. segments: one per distinct key = one per (batch, row).
//
//   data phase, batch after batch:
//     gather  one lane group per sample loads U_b[u] and the K+1 context rows
//             (staged in shared memory), forms s_j = U_b[u].Ctx_b[y_j],
//             g_j = eta_b (1 - sigma(s_j)) for the positive and
//             -eta_b alpha_neg sigma(s_j) for the negatives (Algorithm 1), and
//             writes the per-row gradient contributions to a delta slab:
//             slot 0: sum_j g_j Ctx_b[y_j]; slot 1+j: g_j U_b[u].
//     apply   one lane group per segment sums its slab entries in sorted
//             order and writes X <- X_b - cnt eta_b lambda X_b + sum, with
//             cnt the number of pair occurrences of the row (Eq. 2-3 summed
//             over the batch as in Eq. 4).  BF16 tables are written back with
//             stochastic rounding.
//
// The order of every floating-point sum is fixed, so results are bitwise
// reproducible.  Two schedules run the same per-sample and per-segment code:
//   LINE_MODE_BATCHED     two launches per batch;
//   LINE_MODE_PERSISTENT  one launch per chunk: every warp walks a fixed
//                         list of work items (batch b's samples, then b's
//                         segments, then b+1's ...) and waits, with bounded
//                         spins, only on the items it depends on.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "line_internal.cuh"
#include "scan.cuh"

namespace line {

// ---------------------------------------------------------------------------
// Row geometry: a row of D values is handled by L lanes, E values per lane,
// moved as 16-byte vectors (4 FP32 or 8 BF16 values).
// ---------------------------------------------------------------------------
template <int D, int DT>
struct Geom {
    static constexpr int VEC = DT == LINE_DTYPE_F32 ? 4 : 8;
    static constexpr int L = (D / VEC) < 32 ? (D / VEC) : 32;
    static constexpr int E = D / L;
    static constexpr int NV = E / VEC;
    static constexpr int GPW = 32 / L;  // lane groups per warp
    static_assert(D % (VEC * L) == 0 && NV >= 1, "unsupported dim");
};

template <int D, int DT>
__device__ __forceinline__ void load_row(const void* table, int64_t row, int lig, float (&v)[Geom<D, DT>::E]) {
    using G = Geom<D, DT>;
    if constexpr (DT == LINE_DTYPE_F32) {
        const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(table) + row * D + lig * G::E);
#pragma unroll
        for (int q = 0; q < G::NV; ++q) {
            const float4 a = ld_cg(p + q);
            v[4 * q] = a.x;
            v[4 * q + 1] = a.y;
            v[4 * q + 2] = a.z;
            v[4 * q + 3] = a.w;
        }
    } else {
        const uint4* p = reinterpret_cast<const uint4*>(reinterpret_cast<const __nv_bfloat16*>(table) + row * D + lig * G::E);
#pragma unroll
        for (int q = 0; q < G::NV; ++q) {
            const uint4 a = ld_cg(p + q);
            const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                v[8 * q + 2 * h] = __uint_as_float(w[h] << 16);
                v[8 * q + 2 * h + 1] = __uint_as_float(w[h] & 0xFFFF0000u);
            }
        }
    }
}

// Store a row part; BF16 uses stochastic rounding with bits from the draw at
// counter (row, t0_lo, t0_hi, 2 | table << 4 | (k / 8) << 8), k the first
// column of the 8-value vector (domain 2, one draw per 8 values).
template <int D, int DT>
__device__ __forceinline__ void store_row(void* table, int64_t row, int lig, const float (&v)[Geom<D, DT>::E],
                                          uint64_t seed, uint64_t t0, uint32_t table_id) {
    using G = Geom<D, DT>;
    if constexpr (DT == LINE_DTYPE_F32) {
        float4* p = reinterpret_cast<float4*>(reinterpret_cast<float*>(table) + row * D + lig * G::E);
#pragma unroll
        for (int q = 0; q < G::NV; ++q) st_cg(p + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
    } else {
        uint4* p = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(table) + row * D + lig * G::E);
#pragma unroll
        for (int q = 0; q < G::NV; ++q) {
            const uint32_t k8 = (uint32_t)((lig * G::E + 8 * q) >> 3);
            const uint4 r = philox4x32_10(make_uint4((uint32_t)row, (uint32_t)t0, (uint32_t)(t0 >> 32),
                                                     2u | (table_id << 4) | (k8 << 8)),
                                          make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
            const uint32_t rw[4] = {r.x, r.y, r.z, r.w};
            uint32_t out[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const uint32_t lo = bf16_sr(v[8 * q + 2 * h], rw[h]);
                const uint32_t hi = bf16_sr(v[8 * q + 2 * h + 1], rw[h] >> 16);
                out[h] = lo | (hi << 16);
            }
            st_cg(p + q, make_uint4(out[0], out[1], out[2], out[3]));
        }
    }
}

template <int L>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = L / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Sort item value: (sample within the chunk) << kSlotBits | slot.
constexpr uint32_t kSlotBits = 6;
constexpr uint32_t kSlotMask = (1u << kSlotBits) - 1u;

// ---------------------------------------------------------------------------
// Kernel parameters shared by the data-phase kernels.
// ---------------------------------------------------------------------------
struct DataParams {
    void* U;
    void* C;       // order 2 context table; == U for order 1
    int order, K;  // records have K+2 entries
    int64_t n_nodes;
    uint32_t row_bits;
    const int32_t* rec;        // [chunk samples][K+2]
    const uint64_t* items;     // sorted (key << 32 | value)
    const uint32_t* seg_start; // [n_segs + 1]
    const uint32_t* batch_seg; // [n_batches + 1]
    float* slab;               // [chunk samples][K+2][D]
    uint64_t t_chunk;          // global index of the chunk's first sample
    int64_t chunk_samples;
    int64_t batch;
    int n_batches;
    uint64_t seed;
    const float* eta;  // [n_batches] learning rate of each batch (FP32)
    float lambda, alpha_neg;
    uint32_t* status;
    // persistent schedule
    uint32_t* sample_done;  // [chunk samples] generation flags
    uint32_t* seg_done;     // [chunk segments] generation flags
    uint32_t* batch_applied;  // [n_batches] count of applied segments
    const int32_t* prev_seg;  // [chunk samples][K+2]: segment of the same row in the previous batch, or -1
    const uint64_t* item_base;  // [n_batches + 1] first work item of each batch
    uint32_t gen;
    int64_t spin_limit;
    uint32_t* abort_word;
};

// ---------------------------------------------------------------------------
// Per-sample work: gather, dots, gradient scalars, slab contributions.
// ctx_stage: this warp's shared staging area, (K+1) x 32 lanes x E.
// The record's ids are read by the group's lanes in one go and broadcast, and
// the context rows are loaded CH at a time so their loads are in flight
// together.
// ---------------------------------------------------------------------------
template <int L>
__device__ __forceinline__ uint32_t group_mask(int grp) {
    return L == 32 ? 0xFFFFFFFFu : (((1u << L) - 1u) << (grp * L));
}

template <int D, int DT>
__device__ __forceinline__ void sample_item(const DataParams& p, int64_t s_local, int lig, int lane, bool active,
                                            float eta, float* ctx_stage) {
    using G = Geom<D, DT>;
    constexpr int CH = G::E <= 4 ? 4 : 2;  // context rows in flight per lane
    const int R = p.K + 2;
    const int32_t* rec = p.rec + (active ? s_local : 0) * R;
    const uint32_t gm = group_mask<G::L>(lane / G::L);
    // lane l of the group holds rec[l] (and rec[l + L], ... for small groups)
    const int32_t r0 = (active && lig < R) ? rec[lig] : 0;
    const int32_t u = __shfl_sync(gm, r0, 0, G::L);
    float xu[G::E];
    load_row<D, DT>(p.U, u, lig, xu);
    for (int j0 = 0; j0 <= p.K; j0 += CH) {
        float c[CH][G::E];
#pragma unroll
        for (int jj = 0; jj < CH; ++jj) {
            const int j = j0 + jj;
            const int idx = 1 + j;  // record entry of context row j
            int32_t y = __shfl_sync(gm, r0, idx % G::L, G::L);
            if (idx >= G::L) y = (active && j <= p.K) ? rec[idx] : 0;
            if (j > p.K) y = 0;
            if (j <= p.K) load_row<D, DT>(p.C, y, lig, c[jj]);
        }
#pragma unroll
        for (int jj = 0; jj < CH; ++jj) {
            const int j = j0 + jj;
            if (j <= p.K) {
                float4* st = reinterpret_cast<float4*>(ctx_stage + (j * 32 + lane) * G::E);
#pragma unroll
                for (int q = 0; q < G::E / 4; ++q)
                    st[q] = make_float4(c[jj][4 * q], c[jj][4 * q + 1], c[jj][4 * q + 2], c[jj][4 * q + 3]);
            }
        }
    }
    float du[G::E];
#pragma unroll
    for (int e = 0; e < G::E; ++e) du[e] = 0.0f;
    float* slab = p.slab + (active ? s_local : 0) * (int64_t)R * D + lig * G::E;
    for (int j = 0; j <= p.K; ++j) {
        float c[G::E];
        const float4* ld = reinterpret_cast<const float4*>(ctx_stage + (j * 32 + lane) * G::E);
#pragma unroll
        for (int q = 0; q < G::E / 4; ++q) {
            const float4 a = ld[q];
            c[4 * q] = a.x;
            c[4 * q + 1] = a.y;
            c[4 * q + 2] = a.z;
            c[4 * q + 3] = a.w;
        }
        float part = 0.0f;
#pragma unroll
        for (int e = 0; e < G::E; ++e) part = fmaf(xu[e], c[e], part);
        const float s = group_sum<G::L>(part);
        const float sig = 1.0f / (1.0f + expf(-s));
        const float g = j == 0 ? eta * (1.0f - sig) : -eta * p.alpha_neg * sig;
#pragma unroll
        for (int e = 0; e < G::E; ++e) du[e] = fmaf(g, c[e], du[e]);
        if (active) {
            float4* dst = reinterpret_cast<float4*>(slab + (int64_t)(1 + j) * D);
#pragma unroll
            for (int q = 0; q < G::E / 4; ++q)
                st_cg(dst + q, make_float4(g * xu[4 * q], g * xu[4 * q + 1], g * xu[4 * q + 2], g * xu[4 * q + 3]));
        }
    }
    if (active) {
        float4* dst = reinterpret_cast<float4*>(slab);
#pragma unroll
        for (int q = 0; q < G::E / 4; ++q) st_cg(dst + q, make_float4(du[4 * q], du[4 * q + 1], du[4 * q + 2], du[4 * q + 3]));
    }
}

// ---------------------------------------------------------------------------
// Per-segment work: fixed-order sum of the slab entries of one (batch, row)
// and the write-back.  The group's lanes read the entries' values (and, in
// the persistent schedule, wait on their samples) in parallel, L at a time;
// the slab loads of PF entries are then in flight together and are added in
// sorted order.  Returns false when a bounded wait ran out.
// ---------------------------------------------------------------------------
template <int D, int DT>
__device__ __forceinline__ bool segment_item(const DataParams& p, uint32_t seg, int lig, int lane, bool active,
                                             float eta, uint64_t t0, bool wait_samples) {
    using G = Geom<D, DT>;
    constexpr int PF = G::E <= 4 ? 4 : 2;
    const uint32_t gm = group_mask<G::L>(lane / G::L);
    const uint32_t begin = active ? p.seg_start[seg] : 0u, end = active ? p.seg_start[seg + 1] : 0u;
    const int R = p.K + 2;
    float acc[G::E];
#pragma unroll
    for (int e = 0; e < G::E; ++e) acc[e] = 0.0f;
    int cnt = 0;
    uint32_t key = 0;
    bool ok = true;
    for (uint32_t base = begin; base < end; base += G::L) {
        const uint32_t i = base + (uint32_t)lig;
        const bool have = i < end;
        const uint64_t item = have ? p.items[i] : 0ull;
        if (base == begin) key = __shfl_sync(gm, (uint32_t)(item >> 32), 0, G::L);
        const uint32_t v = (uint32_t)item;
        if (wait_samples && have && ok)
            ok = wait_geq(p.sample_done + (v >> kSlotBits), p.gen, p.spin_limit, p.abort_word);
        const int m = (int)min((uint32_t)G::L, end - base);
        __syncwarp(gm);
        for (int k0 = 0; k0 < m; k0 += PF) {
            float4 buf[PF][G::E / 4];
#pragma unroll
            for (int kk = 0; kk < PF; ++kk) {
                const uint32_t vk = __shfl_sync(gm, v, (k0 + kk) % G::L, G::L);
                if (k0 + kk < m) {
                    const uint32_t slot = vk & kSlotMask;
                    const int64_t entry = (int64_t)(vk >> kSlotBits) * R + slot;
                    const float4* src = reinterpret_cast<const float4*>(p.slab + entry * D + lig * G::E);
#pragma unroll
                    for (int q = 0; q < G::E / 4; ++q) buf[kk][q] = ld_cg(src + q);
                    cnt += slot == 0 ? p.K + 1 : 1;
                }
            }
#pragma unroll
            for (int kk = 0; kk < PF; ++kk) {
                if (k0 + kk < m) {
#pragma unroll
                    for (int q = 0; q < G::E / 4; ++q) {
                        acc[4 * q] += buf[kk][q].x;
                        acc[4 * q + 1] += buf[kk][q].y;
                        acc[4 * q + 2] += buf[kk][q].z;
                        acc[4 * q + 3] += buf[kk][q].w;
                    }
                }
            }
        }
    }
    if (wait_samples && !__all_sync(gm, ok)) return false;
    if (!active) return true;
    const uint32_t rowid = key & ((1u << p.row_bits) - 1u);
    const bool is_c = p.order == 2 && rowid >= (uint32_t)p.n_nodes;
    void* table = is_c ? p.C : p.U;
    const int64_t row = is_c ? (int64_t)rowid - p.n_nodes : (int64_t)rowid;
    float x[G::E];
    load_row<D, DT>(table, row, lig, x);
    const float decay = (float)cnt * (eta * p.lambda);
#pragma unroll
    for (int e = 0; e < G::E; ++e) x[e] = fmaf(-decay, x[e], x[e]) + acc[e];
    store_row<D, DT>(table, row, lig, x, p.seed, t0, is_c ? 1u : 0u);
    return true;
}

// ---------------------------------------------------------------------------
// Batched schedule: one launch per phase per batch.
// ---------------------------------------------------------------------------
constexpr int kMaxWarps = 16;
constexpr size_t kMaxSmem = 200 * 1024;

template <int D, int DT>
__global__ void __launch_bounds__(kMaxWarps * 32) k_gather(DataParams p, int b) {
    using G = Geom<D, DT>;
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G::L, lig = lane % G::L;
    const int64_t s_begin = (int64_t)b * p.batch;
    const int64_t s_end = min(s_begin + p.batch, p.chunk_samples);
    const int64_t s_local = s_begin + ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * G::GPW + grp;
    const float eta = p.eta[b];
    float* stage = smem + (size_t)warp * (p.K + 1) * 32 * G::E;
    sample_item<D, DT>(p, s_local, lig, lane, s_local < s_end, eta, stage);
}

template <int D, int DT>
__global__ void __launch_bounds__(kMaxWarps * 32) k_apply(DataParams p, int b) {
    using G = Geom<D, DT>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G::L, lig = lane % G::L;
    const uint32_t seg_begin = p.batch_seg[b], seg_end = p.batch_seg[b + 1];
    const int64_t s_begin = (int64_t)b * p.batch;
    const uint64_t t0 = p.t_chunk + (uint64_t)s_begin;
    const float eta = p.eta[b];
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x >> 5) * G::GPW;
    // every group of the warp runs the same number of iterations (shuffles)
    const int64_t first = seg_begin + ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * G::GPW;
    for (int64_t sg0 = first; sg0 < seg_end; sg0 += groups) {
        const int64_t sg = sg0 + grp;
        segment_item<D, DT>(p, (uint32_t)sg, lig, lane, sg < seg_end, eta, t0, false);
    }
}

// ---------------------------------------------------------------------------
// Persistent schedule: one cooperative launch per chunk.  Work items in a
// fixed order - batch 0's sample items, batch 0's segment items, batch 1's
// sample items, ... - are dealt round robin to the warps; every warp walks
// its items in increasing order.  An item waits only on items earlier in that
// order, so the earliest unfinished item can always run (all warps are
// resident): the schedule cannot deadlock, and every wait is bounded anyway.
//   sample item (batch b): rows it reads must hold their values after the
//     last batch that touched them: for a row of batch b-1 it waits on that
//     segment's flag; batches b-2 and b-3 must be fully applied (by
//     induction this covers every earlier batch).
//   segment item (batch b): waits for the sample items of its entries (they
//     wrote the slab entries and are the only readers of the row's
//     batch-start value).
// ---------------------------------------------------------------------------
constexpr int kPersistThreads = 256;   // 8 warps per block
constexpr int kPersistMinBlocks = 3;   // <= 85 registers: 24 warps per SM

__device__ __forceinline__ bool batch_applied_ok(const DataParams& p, int bb) {
    if (bb < 0) return true;
    const uint32_t need = p.batch_seg[bb + 1] - p.batch_seg[bb];
    return wait_geq(p.batch_applied + bb, need, p.spin_limit, p.abort_word);
}

__device__ __forceinline__ void fail_abort(const DataParams& p) {
    atomicOr(p.status, DEV_ERR_TIMEOUT);
    atomicExch(p.abort_word, 1u);
}

template <int D, int DT>
__global__ void __launch_bounds__(kPersistThreads, kPersistMinBlocks) k_persistent(DataParams p) {
    using G = Geom<D, DT>;
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G::L, lig = lane % G::L;
    const int wpb = blockDim.x >> 5;
    const int R = p.K + 2;
    float* stage = smem + (size_t)warp * (p.K + 1) * 32 * G::E;
    const uint64_t W = (uint64_t)gridDim.x * wpb;
    const uint64_t total = p.item_base[p.n_batches];
    int b = 0;
    int checked_b = -1;
    for (uint64_t t = (uint64_t)blockIdx.x * wpb + warp; t < total; t += W) {
        while (t >= p.item_base[b + 1]) ++b;
        if (*(volatile uint32_t*)p.abort_word) return;
        const uint64_t local = t - p.item_base[b];
        const int64_t s_begin = (int64_t)b * p.batch;
        const int64_t nb = min((int64_t)p.batch, p.chunk_samples - s_begin);
        const uint64_t nA = (uint64_t)((nb + G::GPW - 1) / G::GPW);
        const uint64_t t0 = p.t_chunk + (uint64_t)s_begin;
        const float eta = p.eta[b];
        if (local < nA) {
            if (checked_b != b) {
                if (!batch_applied_ok(p, b - 2) || !batch_applied_ok(p, b - 3)) {
                    fail_abort(p);
                    return;
                }
                checked_b = b;
            }
            const int64_t s_local = s_begin + (int64_t)local * G::GPW + grp;
            const bool active = s_local < s_begin + nb;
            bool ok = true;
            if (active) {
                for (int k = lig; k < R; k += G::L) {
                    const int32_t ps = p.prev_seg[s_local * R + k];
                    if (ps >= 0 && !wait_geq(p.seg_done + ps, p.gen, p.spin_limit, p.abort_word)) ok = false;
                }
            }
            if (!__all_sync(0xFFFFFFFFu, ok)) {
                fail_abort(p);
                return;
            }
            sample_item<D, DT>(p, s_local, lig, lane, active, eta, stage);
            __syncwarp();
            if (active && lig == 0) st_release(p.sample_done + s_local, p.gen);
        } else {
            const uint32_t seg = p.batch_seg[b] + (uint32_t)((local - nA) * G::GPW) + grp;
            const bool active = seg < p.batch_seg[b + 1];
            const bool ok = segment_item<D, DT>(p, seg, lig, lane, active, eta, t0, true);
            if (!__all_sync(0xFFFFFFFFu, ok)) {
                fail_abort(p);
                return;
            }
            // the group's row stores are ordered before the flag by the warp
            // barrier; the release store publishes them
            __syncwarp();
            if (active && lig == 0) {
                st_release(p.seg_done + seg, p.gen);
                red_release_add(p.batch_applied + b, 1u);
            }
        }
    }
}

// eta[b] = lr0 (schedule 0) or lr0 * max(1 - t0/T, floor) (schedule 1) for
// the batch starting at global sample t0 = t_chunk + b * batch; FP64 once per
// batch, used as FP32.
__global__ void k_batch_eta(int n_batches, uint64_t t_chunk, int64_t batch, double lr0, int schedule, double floor_frac,
                            uint64_t total, float* __restrict__ eta) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_batches) return;
    double f = 1.0;
    if (schedule == 1) {
        f = 1.0 - (double)(t_chunk + (uint64_t)b * (uint64_t)batch) / (double)total;
        if (f < floor_frac) f = floor_frac;
    }
    eta[b] = (float)(lr0 * f);
}

// item_base[b] = first work item of batch b (sample items then segment items).
__global__ void k_item_base(const uint32_t* __restrict__ batch_seg, int n_batches, int64_t batch,
                            int64_t chunk_samples, int gpw, uint64_t* __restrict__ item_base) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    uint64_t acc = 0;
    for (int b = 0; b < n_batches; ++b) {
        item_base[b] = acc;
        const int64_t nb = min(batch, chunk_samples - (int64_t)b * batch);
        acc += (uint64_t)((nb + gpw - 1) / gpw);
        acc += (uint64_t)((batch_seg[b + 1] - batch_seg[b] + gpw - 1) / gpw);
    }
    item_base[n_batches] = acc;
}

// prev_seg[(sample, slot)] = segment of the same row in the previous batch of
// the chunk, or -1.  One thread per segment: binary search among the previous
// batch's segment keys, then written for every entry of the segment.
__global__ void k_prev_seg(const uint64_t* __restrict__ items, const uint32_t* __restrict__ seg_start,
                           const uint32_t* n_segs_p, const uint32_t* __restrict__ batch_seg, uint32_t row_bits,
                           uint32_t R, int32_t* __restrict__ prev_seg) {
    const uint32_t n_segs = *n_segs_p;
    const uint32_t mask = (1u << row_bits) - 1u;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n_segs; j += gridDim.x * blockDim.x) {
        const uint32_t key = (uint32_t)(items[seg_start[j]] >> 32);
        const uint32_t b = key >> row_bits;
        int32_t ps = -1;
        if (b > 0) {
            const uint32_t want = ((b - 1) << row_bits) | (key & mask);
            uint32_t lo = batch_seg[b - 1], hi = batch_seg[b];
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if ((uint32_t)(items[seg_start[mid]] >> 32) < want) lo = mid + 1;
                else hi = mid;
            }
            if (lo < batch_seg[b] && (uint32_t)(items[seg_start[lo]] >> 32) == want) ps = (int32_t)lo;
        }
        for (uint32_t i = seg_start[j]; i < seg_start[j + 1]; ++i) {
            const uint32_t v = (uint32_t)items[i];
            prev_seg[(v >> kSlotBits) * R + (v & kSlotMask)] = ps;
        }
    }
}

// ---------------------------------------------------------------------------
// Pre-pass kernels.
// ---------------------------------------------------------------------------
struct PrepassParams {
    const int32_t* src;
    const int32_t* dst;
    const uint2* edge_tab;
    const uint2* neg_tab;
    int64_t n_arcs, n_nodes;
    uint64_t seed;
    uint64_t t_chunk;
    int64_t chunk_samples;
    int64_t batch;
    int K, order;
    uint32_t row_bits;
    int32_t* rec;
    uint64_t* items;
};

__device__ __forceinline__ uint64_t make_item(uint32_t batch, uint32_t row_bits, uint32_t rowid, uint32_t s_local,
                                              uint32_t slot) {
    return ((uint64_t)((batch << row_bits) | rowid) << 32) | ((s_local << kSlotBits) | slot);
}

__global__ void k_chunk_draws(PrepassParams p) {
    const uint32_t C1 = (uint32_t)p.K + 1u, R = (uint32_t)p.K + 2u;
    const uint32_t total = (uint32_t)p.chunk_samples * C1;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const uint32_t s = q / C1;
        const uint32_t c = q - s * C1;
        const uint32_t b = s / (uint32_t)p.batch;
        const uint4 w = draw_words(p.seed, 0u, p.t_chunk + (uint64_t)s, c);
        const uint32_t ctx_off = p.order == 2 ? (uint32_t)p.n_nodes : 0u;
        const uint32_t base = s * R;
        if (c == 0) {
            const uint32_t e = alias_pick(p.edge_tab, (uint64_t)p.n_arcs, w);
            const int32_t u = __ldg(p.src + e), v = __ldg(p.dst + e);
            p.rec[base] = u;
            p.rec[base + 1] = v;
            p.items[base] = make_item(b, p.row_bits, (uint32_t)u, s, 0u);
            p.items[base + 1] = make_item(b, p.row_bits, (uint32_t)v + ctx_off, s, 1u);
        } else {
            const uint32_t y = alias_pick(p.neg_tab, (uint64_t)p.n_nodes, w);
            p.rec[base + 1 + c] = (int32_t)y;
            p.items[base + 1 + c] = make_item(b, p.row_bits, y + ctx_off, s, 1u + c);
        }
    }
}

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 16;
constexpr int kRsTile = kRsThreads * kRsRounds;  // 4096 items
constexpr int kRsBits = 8;
constexpr int kRsBins = 1 << kRsBits;

__global__ void __launch_bounds__(kRsThreads) k_radix_hist(const uint64_t* __restrict__ in, int64_t n, int shift,
                                                           uint32_t* __restrict__ hist, int ntiles) {
    __shared__ uint32_t cnt[kRsBins];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
    for (int r = 0; r < kRsRounds; ++r) {
        const int64_t i = base + r * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(uint32_t)(in[i] >> shift) & (kRsBins - 1)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

struct GenU32 {
    const uint32_t* a;
    __device__ uint32_t operator()(int64_t i) const { return a[i]; }
};
struct OutExcl32 {
    uint32_t* a;
    __device__ void operator()(int64_t i, uint32_t excl, uint32_t) const { a[i] = excl; }
};

// Stable scatter: warp w owns items [tile + 512 w, +512) and ranks them in 16
// rounds of 32 (index order); per-digit warp counts then give every item its
// position among equal digits of the tile.
__global__ void __launch_bounds__(kRsThreads) k_radix_scatter(const uint64_t* __restrict__ in,
                                                              uint64_t* __restrict__ out, int64_t n, int shift,
                                                              const uint32_t* __restrict__ offs, int ntiles) {
    __shared__ uint32_t wcnt[kRsWarps][kRsBins];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)warp * (kRsRounds * 32);
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t key[kRsRounds];
    uint32_t dig[kRsRounds], rank[kRsRounds];
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool valid = i < n;
        key[r] = valid ? in[i] : 0ull;
        const uint32_t d = valid ? (uint32_t)(key[r] >> shift) & (kRsBins - 1) : 0xFFFFu;
        dig[r] = d;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t before = valid ? wcnt[warp][d] : 0u;
        rank[r] = before + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) {
            const uint32_t c = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const int64_t i = base + r * 32 + lane;
        if (i < n) {
            const uint32_t d = dig[r];
            out[offs[(int64_t)d * ntiles + blockIdx.x] + wcnt[warp][d] + rank[r]] = key[r];
        }
    }
}

struct GenHead {
    const uint64_t* items;
    __device__ uint32_t operator()(int64_t i) const {
        return (i == 0 || (items[i] >> 32) != (items[i - 1] >> 32)) ? 1u : 0u;
    }
};
struct OutSegStart {
    const uint64_t* items;
    uint32_t* seg_start;
    int64_t n;
    uint32_t* n_segs;
    __device__ void operator()(int64_t i, uint32_t excl, uint32_t incl) const {
        if (i == 0 || (items[i] >> 32) != (items[i - 1] >> 32)) seg_start[excl] = (uint32_t)i;
        if (i == n - 1) {
            seg_start[incl] = (uint32_t)n;
            *n_segs = incl;
        }
    }
};

// batch_seg[b] = first segment of batch b; batch_seg[n_batches] = n_segs.
__global__ void k_batch_seg(const uint64_t* __restrict__ items, const uint32_t* __restrict__ seg_start,
                            const uint32_t* n_segs_p, uint32_t row_bits, int n_batches, uint32_t* __restrict__ batch_seg) {
    const uint32_t n_segs = *n_segs_p;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n_segs; j += gridDim.x * blockDim.x) {
        const int bj = (int)((uint32_t)(items[seg_start[j]] >> 32) >> row_bits);
        const int bp = j ? (int)((uint32_t)(items[seg_start[j - 1]] >> 32) >> row_bits) : -1;
        for (int b = bp + 1; b <= bj; ++b) batch_seg[b] = j;
        if (j + 1 == n_segs)
            for (int b = bj + 1; b <= n_batches; ++b) batch_seg[b] = n_segs;
    }
}

// ---------------------------------------------------------------------------
// Workspace.
// ---------------------------------------------------------------------------
struct Buf {
    void* p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e == cudaSuccess) cap = bytes;
        return e;
    }
    ~Buf() {
        if (p) cudaFree(p);
    }
};

struct TrainWorkspace {
    Buf rec, items0, items1, hist, scan_tiles, seg_start, batch_seg, counters, slab;
    Buf sample_done, seg_done, batch_applied, prev_seg, item_base, eta;
    std::vector<cudaEvent_t> events;  // timing events, three per chunk
    uint32_t gen = 0;
    cudaError_t event(size_t i, cudaEvent_t* out) {
        while (events.size() <= i) {
            cudaEvent_t e;
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return r;
            events.push_back(e);
        }
        *out = events[i];
        return cudaSuccess;
    }
};

TrainWorkspace* workspace_create() { return new TrainWorkspace(); }
void workspace_destroy(TrainWorkspace* ws) {
    if (!ws) return;
    for (auto e : ws->events) cudaEventDestroy(e);
    delete ws;
}

static uint32_t bits_for(uint64_t v) {  // bits to hold values 0..v-1
    uint32_t b = 1;
    while ((1ull << b) < v) ++b;
    return b;
}

template <int D, int DT>
static cudaError_t launch_data_batched(const DataParams& p, int warps_per_block, cudaStream_t s) {
    using G = Geom<D, DT>;
    // staging: (K+1) context rows x 32 lanes x E floats per warp; at most
    // kMaxSmem per block, at most kMaxWarps warps
    const size_t per_warp = (size_t)(p.K + 1) * 32 * G::E * sizeof(float);
    int wpb = warps_per_block > 0 ? warps_per_block : 8;
    wpb = std::min<int>(wpb, kMaxWarps);
    wpb = std::max<int>(1, std::min<int>(wpb, (int)(kMaxSmem / per_warp)));
    const size_t smem = (size_t)wpb * per_warp;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_gather<D, DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
        attr_set = true;
    }
    const int64_t per_block = (int64_t)wpb * G::GPW;
    for (int b = 0; b < p.n_batches; ++b) {
        const int64_t nb = std::min<int64_t>(p.batch, p.chunk_samples - (int64_t)b * p.batch);
        const unsigned g1 = (unsigned)((nb + per_block - 1) / per_block);
        k_gather<D, DT><<<g1, wpb * 32, smem, s>>>(p, b);
        const int64_t max_segs = nb * (p.K + 2);
        const unsigned g2 = (unsigned)std::min<int64_t>((max_segs + per_block - 1) / per_block, 152 * 16);
        k_apply<D, DT><<<g2, wpb * 32, 0, s>>>(p, b);
    }
    return cudaGetLastError();
}

template <int D, int DT>
static cudaError_t launch_data_persistent(const DataParams& p, int warps_per_block, cudaStream_t s) {
    using G = Geom<D, DT>;
    const size_t per_warp = (size_t)(p.K + 1) * 32 * G::E * sizeof(float);
    int wpb = warps_per_block > 0 ? warps_per_block : 8;
    wpb = std::min<int>(wpb, kPersistThreads / 32);
    wpb = std::max<int>(1, std::min<int>(wpb, (int)(kMaxSmem / per_warp)));
    const size_t smem = (size_t)wpb * per_warp;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_persistent<D, DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
        attr_set = true;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent<D, DT>, wpb * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    DataParams pc = p;
    void* args[] = {&pc};
    return cudaLaunchCooperativeKernel((const void*)k_persistent<D, DT>, dim3((unsigned)(per_sm * sms)),
                                       dim3((unsigned)(wpb * 32)), args, smem, s);
}

using LaunchFn = cudaError_t (*)(const DataParams&, int, cudaStream_t);

static LaunchFn pick_persistent(int dim, int dtype) {
#define LINE_PICK(DD)                                                                          \
    if (dim == DD) return dtype == LINE_DTYPE_F32 ? launch_data_persistent<DD, LINE_DTYPE_F32> \
                                                  : launch_data_persistent<DD, LINE_DTYPE_BF16>;
    LINE_PICK(16)
    LINE_PICK(32)
    LINE_PICK(64)
    LINE_PICK(128)
    LINE_PICK(256)
#undef LINE_PICK
    return nullptr;
}

static int groups_per_warp(int dim, int dtype) {
    const int vec = dtype == LINE_DTYPE_F32 ? 4 : 8;
    const int L = std::min(32, dim / vec);
    return 32 / L;
}

static LaunchFn pick_batched(int dim, int dtype) {
#define LINE_PICK(DD)                                                                       \
    if (dim == DD) return dtype == LINE_DTYPE_F32 ? launch_data_batched<DD, LINE_DTYPE_F32> \
                                                  : launch_data_batched<DD, LINE_DTYPE_BF16>;
    LINE_PICK(16)
    LINE_PICK(32)
    LINE_PICK(64)
    LINE_PICK(128)
    LINE_PICK(256)
#undef LINE_PICK
    return nullptr;
}

cudaError_t train_run(const TrainArgs& a, TrainWorkspace* ws, uint32_t* status, TrainTimes* times, cudaStream_t s,
                      std::string* err) {
    const int R = a.K + 2;
    const uint64_t n_samples = a.t_end - a.t_begin;
    if (n_samples == 0) return cudaSuccess;
    const uint64_t rows_space = a.order == 2 ? 2ull * (uint64_t)a.n_nodes : (uint64_t)a.n_nodes;
    const uint32_t row_bits = bits_for(rows_space);
    if (row_bits > 31) {
        *err = "too many nodes for 32-bit sort keys";
        return cudaErrorInvalidValue;
    }
    // batches per chunk: about 2^18 samples, limited by the key bits and by
    // 32-bit item values (chunk samples * (K+2) < 2^32)
    int64_t nb_max = (int64_t)1 << (32 - row_bits);
    int64_t nb = a.chunk_batches > 0 ? a.chunk_batches : std::max<int64_t>(1, (int64_t(1) << 18) / a.batch);
    nb = std::min(nb, nb_max);
    // item values hold the chunk sample in 32 - kSlotBits bits
    while (nb > 1 && ((uint64_t)nb * (uint64_t)a.batch * (uint64_t)R >= (1ull << 31) ||
                      (uint64_t)nb * (uint64_t)a.batch > (1ull << (32 - kSlotBits))))
        nb >>= 1;
    const uint64_t total_batches = (n_samples + a.batch - 1) / a.batch;
    nb = (int64_t)std::min<uint64_t>((uint64_t)nb, total_batches);
    const uint32_t batch_bits = bits_for((uint64_t)nb);
    const uint32_t key_bits = batch_bits + row_bits;
    const int64_t max_chunk = nb * a.batch;
    const int64_t max_items = max_chunk * R;
    const int ntiles = (int)((max_items + kRsTile - 1) / kRsTile);

    cudaError_t e;
    auto ensure = [&](Buf& b, size_t bytes) -> bool {
        if ((e = b.ensure(bytes)) != cudaSuccess) {
            *err = "device allocation failed (training scratch)";
            return false;
        }
        return true;
    };
    if (!ensure(ws->rec, sizeof(int32_t) * max_items) || !ensure(ws->items0, sizeof(uint64_t) * max_items) ||
        !ensure(ws->items1, sizeof(uint64_t) * max_items) ||
        !ensure(ws->hist, sizeof(uint32_t) * (size_t)kRsBins * ntiles) ||
        !ensure(ws->scan_tiles, sizeof(uint32_t) * (scan_tiles((int64_t)kRsBins * ntiles + max_items) + 2)) ||
        !ensure(ws->seg_start, sizeof(uint32_t) * (max_items + 1)) ||
        !ensure(ws->batch_seg, sizeof(uint32_t) * (nb + 1)) || !ensure(ws->counters, 256) ||
        !ensure(ws->eta, sizeof(float) * (nb + 1)) ||
        !ensure(ws->slab, sizeof(float) * (size_t)max_items * a.dim))
        return e;
    const bool persistent = a.mode == LINE_MODE_PERSISTENT;
    if (persistent) {
        if (!ensure(ws->prev_seg, sizeof(int32_t) * max_items) || !ensure(ws->item_base, sizeof(uint64_t) * (nb + 1)) ||
            !ensure(ws->batch_applied, sizeof(uint32_t) * (nb + 1)))
            return e;
        // generation flags start at zero and are never reset: a chunk's
        // flags are "done" when they equal its generation number
        const size_t need_s = sizeof(uint32_t) * max_chunk, need_g = sizeof(uint32_t) * (max_items + 1);
        if (ws->sample_done.cap < need_s) {
            if (!ensure(ws->sample_done, need_s)) return e;
            if ((e = cudaMemsetAsync(ws->sample_done.p, 0, need_s, s)) != cudaSuccess) return e;
            ws->gen = 0;
        }
        if (ws->seg_done.cap < need_g) {
            if (!ensure(ws->seg_done, need_g)) return e;
            if ((e = cudaMemsetAsync(ws->seg_done.p, 0, need_g, s)) != cudaSuccess) return e;
            if ((e = cudaMemsetAsync(ws->sample_done.p, 0, ws->sample_done.cap, s)) != cudaSuccess) return e;
            ws->gen = 0;
        }
    }
    LaunchFn data = persistent ? pick_persistent(a.dim, a.dtype) : pick_batched(a.dim, a.dtype);
    if (!data) {
        *err = "unsupported dim";
        return cudaErrorInvalidValue;
    }

    PrepassParams pp;
    pp.src = a.src;
    pp.dst = a.dst;
    pp.edge_tab = a.edge_tab;
    pp.neg_tab = a.neg_tab;
    pp.n_arcs = a.n_arcs;
    pp.n_nodes = a.n_nodes;
    pp.seed = a.seed;
    pp.batch = a.batch;
    pp.K = a.K;
    pp.order = a.order;
    pp.row_bits = row_bits;
    pp.rec = (int32_t*)ws->rec.p;

    DataParams dp{};
    dp.U = nullptr;
    dp.order = a.order;
    dp.K = a.K;
    dp.n_nodes = a.n_nodes;
    dp.row_bits = row_bits;
    dp.rec = (const int32_t*)ws->rec.p;
    dp.seg_start = (const uint32_t*)ws->seg_start.p;
    dp.batch_seg = (const uint32_t*)ws->batch_seg.p;
    dp.slab = (float*)ws->slab.p;
    dp.batch = a.batch;
    dp.seed = a.seed;
    dp.eta = (const float*)ws->eta.p;
    dp.lambda = (float)a.lambda;
    dp.alpha_neg = (float)a.alpha_neg;
    dp.status = status;
    dp.U = a.U;
    dp.C = a.order == 2 ? a.C : a.U;

    uint32_t* n_segs_dev = (uint32_t*)ws->counters.p;
    uint32_t* abort_word = (uint32_t*)ws->counters.p + 16;
    dp.sample_done = (uint32_t*)ws->sample_done.p;
    dp.seg_done = (uint32_t*)ws->seg_done.p;
    dp.batch_applied = (uint32_t*)ws->batch_applied.p;
    dp.prev_seg = (const int32_t*)ws->prev_seg.p;
    dp.item_base = (const uint64_t*)ws->item_base.p;
    dp.spin_limit = a.spin_limit;
    dp.abort_word = abort_word;
    size_t n_ev = 0;
    struct ChunkRec {
        int64_t samples;
        int batches;
    };
    std::vector<ChunkRec> chunk_log;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr, ev_c = nullptr;
    for (uint64_t t = a.t_begin; t < a.t_end; t += (uint64_t)max_chunk) {
        const int64_t cs = (int64_t)std::min<uint64_t>((uint64_t)max_chunk, a.t_end - t);
        const int cb = (int)((cs + a.batch - 1) / a.batch);
        const int64_t n_items = cs * R;
        if (a.timing) {
            if ((e = ws->event(n_ev, &ev_a)) != cudaSuccess) return e;
            cudaEventRecord(ev_a, s);
        }
        // 1. draws
        pp.t_chunk = t;
        pp.chunk_samples = cs;
        pp.items = (uint64_t*)ws->items0.p;
        {
            const int64_t work = cs * (a.K + 1);
            const unsigned g = (unsigned)std::min<int64_t>((work + 255) / 256, 152 * 64);
            k_chunk_draws<<<g, 256, 0, s>>>(pp);
        }
        // 2. stable LSD radix sort by key bits [32, 32 + key_bits)
        uint64_t* in = (uint64_t*)ws->items0.p;
        uint64_t* out = (uint64_t*)ws->items1.p;
        const int tiles = (int)((n_items + kRsTile - 1) / kRsTile);
        uint32_t* hist = (uint32_t*)ws->hist.p;
        for (uint32_t sh = 0; sh < key_bits; sh += kRsBits) {
            k_radix_hist<<<tiles, kRsThreads, 0, s>>>(in, n_items, 32 + (int)sh, hist, tiles);
            if ((e = device_scan<uint32_t>((int64_t)kRsBins * tiles, GenU32{hist}, OutExcl32{hist},
                                           (uint32_t*)ws->scan_tiles.p, s)) != cudaSuccess)
                return e;
            k_radix_scatter<<<tiles, kRsThreads, 0, s>>>(in, out, n_items, 32 + (int)sh, hist, tiles);
            std::swap(in, out);
        }
        // 3. segments
        if ((e = device_scan<uint32_t>(n_items, GenHead{in},
                                       OutSegStart{in, (uint32_t*)ws->seg_start.p, n_items, n_segs_dev},
                                       (uint32_t*)ws->scan_tiles.p, s)) != cudaSuccess)
            return e;
        k_batch_eta<<<(unsigned)((cb + 127) / 128), 128, 0, s>>>(cb, t, a.batch, a.lr0, a.lr_schedule, a.lr_floor,
                                                                 a.lr_total, (float*)ws->eta.p);
        k_batch_seg<<<(unsigned)std::min<int64_t>((n_items + 255) / 256, 152 * 16), 256, 0, s>>>(
            in, (const uint32_t*)ws->seg_start.p, n_segs_dev, row_bits, cb, (uint32_t*)ws->batch_seg.p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (persistent) {
            const unsigned gs = (unsigned)std::min<int64_t>((n_items + 255) / 256, 152 * 16);
            k_prev_seg<<<gs, 256, 0, s>>>(in, (const uint32_t*)ws->seg_start.p, n_segs_dev, (const uint32_t*)ws->batch_seg.p,
                                          row_bits, (uint32_t)R, (int32_t*)ws->prev_seg.p);
            k_item_base<<<1, 32, 0, s>>>((const uint32_t*)ws->batch_seg.p, cb, a.batch, cs,
                                         groups_per_warp(a.dim, a.dtype), (uint64_t*)ws->item_base.p);
            if ((e = cudaMemsetAsync(ws->batch_applied.p, 0, sizeof(uint32_t) * (cb + 1), s)) != cudaSuccess) return e;
            if ((e = cudaMemsetAsync(abort_word, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            dp.gen = ++ws->gen;
        }
        if (a.timing) {
            if ((e = ws->event(n_ev + 1, &ev_b)) != cudaSuccess) return e;
            cudaEventRecord(ev_b, s);
        }
        // data phase
        dp.items = in;
        dp.t_chunk = t;
        dp.chunk_samples = cs;
        dp.n_batches = cb;
        if ((e = data(dp, a.warps_per_block, s)) != cudaSuccess) return e;
        if (a.timing) {
            if ((e = ws->event(n_ev + 2, &ev_c)) != cudaSuccess) return e;
            cudaEventRecord(ev_c, s);
            n_ev += 3;
            chunk_log.push_back({cs, cb});
        }
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (a.timing && n_ev) {
        if ((e = cudaEventSynchronize(ws->events[n_ev - 1])) != cudaSuccess) return e;
        const int64_t passes = (key_bits + kRsBits - 1) / kRsBits;
        for (size_t i = 0; i < chunk_log.size(); ++i) {
            float ms1 = 0, ms2 = 0;
            cudaEventElapsedTime(&ms1, ws->events[3 * i], ws->events[3 * i + 1]);
            cudaEventElapsedTime(&ms2, ws->events[3 * i + 1], ws->events[3 * i + 2]);
            times->prepass_ms += ms1;
            times->update_ms += ms2;
            // draws + per pass (hist, 3 scan launches, scatter) + segment scan (3) + batch_seg
            times->prepass_launches += 1 + 5 * passes + 5 + (persistent ? 2 : 0);
            times->update_launches += persistent ? 1 : 2 * (int64_t)chunk_log[i].batches;
            times->update_samples += (uint64_t)chunk_log[i].samples;
        }
    }
    return cudaSuccess;
}

}  // namespace line
