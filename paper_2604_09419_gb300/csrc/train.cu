// Minibatch-synchronous LINE training on the GPU (Algorithm 1, Eq. 2-4).
//
// A call processes its samples in chunks of whole batches.  Per chunk:
//
//   pre-pass (index work only; it does not read the tables), on its own
//   low-priority stream so that it overlaps the previous chunk's data phase:
//     1. draws: for every sample its arc (u, v) and K negatives, kept as a
//        record (u, v, n_1..n_K), and K+2 items, one per row the sample
//        touches: key = row id, value = (sample, slot).  Slot 0 is U[u];
//        slots 1..K+1 are the context rows Ctx[v], Ctx[n_j] (Ctx = C for
//        second order, U for first order; C rows get ids offset by n).
//     2. per batch, a stable counting sort of the batch's items into 256
//        buckets by a hash of the row id;
//     3. per (batch, bucket), a stable sort by row id, then the segments: runs of equal row = the rows the batch touches,
//        entries in (sample, slot) order.  A segment with one entry is a
//        singleton: its row is read and written by one sample only.  Every
//        (sample, slot) learns its position and its segment; segments with
//        two or more entries ("shared") are listed per batch with their first
//        position, length, row and pair count.
//
//   data phase, batch after batch:
//     gather  one lane group per sample loads U_b[u] and the K+1 context
//             rows (staged in shared memory), forms s_j = U_b[u].Ctx_b[y_j],
//             g_j = eta_b (1 - sigma(s_j)) for the positive and
//             -eta_b alpha_neg sigma(s_j) for the negatives (Algorithm 1).
//             Its contributions are slot 0: sum_j g_j Ctx_b[y_j] for U[u],
//             slot 1+j: g_j U_b[u] for Ctx[y_j].  A singleton row is written
//             back at once (Eq. 2-3); a shared row's contribution goes to the
//             delta slab at its position, so a segment's entries are
//             contiguous.  Positions count from the batch's first item: every
//             batch reuses one slab region, whose lines stay in L2 instead of
//             being written back to DRAM.
//     apply   per shared segment: the entries summed in a fixed chunked
//             order, X <- X_b - cnt eta_b lambda X_b + sum, cnt the number of
//             pair occurrences of the row (the batch-summed update of Eq. 4).
//   BF16 tables are written back with stochastic rounding (random bits from
//   a counter hash of seed, table, row, batch and column group).
//
// The order of every floating-point sum is fixed, so results are bitwise
// reproducible, and a singleton row gets exactly the value the apply step
// would give it.  Two schedules run the same per-sample and per-segment code:
//   LINE_MODE_BATCHED     two launches per batch, chained with programmatic
//                         dependent launch;
//   LINE_MODE_PERSISTENT  one cooperative launch per chunk: resident CTAs
//                         loop over the chunk's batches, rows staged in
//                         shared memory by bulk copies, a grid-wide barrier
//                         after each batch's gather and after its apply.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "bulk.cuh"
#include "line_internal.cuh"
#include "rows.cuh"
#include "scan.cuh"

namespace line {

namespace cg = cooperative_groups;

// Programmatic dependent launch: let the next kernel of the stream start its
// prologue, and wait until the previous kernel's writes are visible.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// A shared segment's entries are summed in chunks of kChunk: partial sums in
// entry order, then the partials in chunk order.  Segments longer than one
// chunk (the hub rows) are summed by a whole CTA in the batched schedule.
constexpr uint32_t kChunk = 8;
constexpr uint32_t kLongBit = 1u << 31;  // in mdesc.y: summed by a CTA

// Sort item value: (sample within the chunk) << kSlotBits | slot.
constexpr uint32_t kSlotBits = 6;
constexpr uint32_t kSlotMask = (1u << kSlotBits) - 1u;
// slot_info.x: sorted position within the batch, bit 31 set for a singleton segment.
constexpr uint32_t kSingleBit = 1u << 31;

// Fibonacci hashing: spreads the hot (low) row ids of skewed graphs.  The
// multiplier is odd, so hrow is a bijection of 32-bit words (inverse
// 0x0E8B2F51); within a batch items are ordered by (hrow(row), index), which
// puts them bucket by bucket (bucket = top 8 bits) and each row's entries
// together in index order.
__device__ __forceinline__ uint32_t hrow(uint32_t row) { return row * 0x9E3779B1u; }
__device__ __forceinline__ uint32_t unhrow(uint32_t h) { return h * 0x0E8B2F51u; }
__device__ __forceinline__ uint32_t bucket_of(uint32_t row) { return hrow(row) >> 24; }

// Rows a batch touches, as a bitmap of 2^kDepLog bits indexed by the top bits
// of hrow(row id) (row ids: U rows 0..n-1, C rows n..2n-1 in second order).
// A row whose bit is clear in batch b's map is not written by batch b, so it
// may be read for batch b+1 while batch b is still running (a false positive
// only delays a read).
constexpr int kDepLog = 18;
constexpr uint32_t kDepWords = 1u << (kDepLog - 5);
__device__ __forceinline__ uint32_t dep_bit(uint32_t rowid) { return hrow(rowid) >> (32 - kDepLog); }

// ---------------------------------------------------------------------------
// Kernel parameters shared by the data-phase kernels.
// ---------------------------------------------------------------------------
struct DataParams {
    void* U;
    void* C;       // order 2 context table; == U for order 1
    int order, K;  // records have K+2 entries
    int apply_warps;  // warps of an apply block (batched schedule)
    int64_t n_nodes;
    uint32_t row_bits;
    const int32_t* rec;      // [chunk samples][K+2]
    const uint2* slot_info;  // [chunk samples][K+2]: {position | singleton bit, segment (first position)}
    const uint4* mdesc;      // [n_batches][mcap] shared segments: {first position, length | long bit, row, pair count}
    const uint32_t* mcount;  // [n_batches]
    uint32_t mcap;
    const uint4* ldesc;      // [n_batches][lcap] long shared segments (also in mdesc, flagged)
    const uint32_t* lcount;  // [n_batches]
    uint32_t lcap;
    float* slab;             // [batch * (K+2)][D], by position within the batch
    const uint32_t* depmap;  // [n_batches][kDepWords] rows each batch touches (bit dep_bit(row id))
    uint64_t t_chunk;        // global index of the chunk's first sample
    const uint64_t* t_chunk_dev;  // when set, the same read from device memory (graph replays)
    int64_t chunk_samples;
    int64_t batch;
    int n_batches;
    uint64_t seed;
    const float* eta;  // [n_batches] learning rate of each batch (FP32)
    float lambda, alpha_neg;
    uint32_t* status;
    // persistent schedule
    uint32_t* gbar;           // grid barrier: {arrivals, completed rounds}, zero at launch
    int slots;                // shared-memory row slots per warp (1 or 2)
    int64_t spin_limit;
    uint32_t* abort_word;
};

// Record entry idx of the group's sample: lane idx % L holds entries
// idx < L in `held`; later ones are read from memory.
__device__ __forceinline__ int32_t shfl_w(uint32_t gm, int32_t v, int src, int w) { return __shfl_sync(gm, v, src, w); }
__device__ __forceinline__ uint2 shfl_w(uint32_t gm, uint2 v, int src, int w) {
    return make_uint2(__shfl_sync(gm, v.x, src, w), __shfl_sync(gm, v.y, src, w));
}

template <int L, typename T>
__device__ __forceinline__ T rec_entry(uint32_t gm, T held, const T* row, int idx, bool active) {
    T v = shfl_w(gm, held, idx % L, L);
    if (idx >= L) v = active ? row[idx] : T{};
    return v;
}

// ---------------------------------------------------------------------------
// Per-sample work.
// ctx_stage: this warp's shared staging area, (K+1) x 32 lanes x E floats.
// ---------------------------------------------------------------------------
// Register-resident gather body for K + 1 <= JB (6 or 8): the K+1 context
// rows stay in registers; the dots, their reductions and the K+1 sigmoids are
// independent chains.  Same arithmetic, in the same order, as the staged
// body.  JB = 6 covers K <= 5 in fewer registers, so that a batch's gather
// leaves room on every SM for the next chunk's pre-pass.
template <int D, int DT, int JB = 8>
__device__ __forceinline__ void sample_body_reg(const DataParams& p, int lig, bool active, float eta, uint64_t t0,
                                                uint32_t gm, int32_t r0, uint2 i0, const int32_t* rec,
                                                const uint2* info) {
    using G = Geom<D, DT>;
    const int32_t u = __shfl_sync(gm, r0, 0, G::L);
    float xu[G::E];
    float c[JB][G::E];
    load_row<D, DT>(p.U, u, lig, xu);
#pragma unroll
    for (int j = 0; j < JB; ++j) {
        const int32_t y = rec_entry<G::L>(gm, r0, rec, 1 + j, active && j <= p.K);
        if (j <= p.K) load_row<D, DT>(p.C, y, lig, c[j]);
    }
    float sj[JB];
#pragma unroll
    for (int j = 0; j < JB; ++j) {
        sj[j] = 0.0f;
#pragma unroll
        for (int e = 0; e < G::E; ++e) sj[j] = fmaf(xu[e], c[j][e], sj[j]);
    }
#pragma unroll
    for (int o = G::L / 2; o >= 1; o >>= 1)
#pragma unroll
        for (int j = 0; j < JB; ++j) sj[j] += __shfl_xor_sync(0xFFFFFFFFu, sj[j], o);
    float g[JB];
#pragma unroll
    for (int j = 0; j < JB; ++j) {
        const float sig = 1.0f / (1.0f + expf(-sj[j]));
        g[j] = j == 0 ? eta * (1.0f - sig) : -eta * p.alpha_neg * sig;
    }
    const uint32_t ctx_table = p.order == 2 ? 1u : 0u;
    const float etalam = eta * p.lambda;
    float du[G::E];
#pragma unroll
    for (int e = 0; e < G::E; ++e) du[e] = 0.0f;
#pragma unroll
    for (int j = 0; j < JB; ++j) {
        if (j > p.K) continue;
#pragma unroll
        for (int e = 0; e < G::E; ++e) du[e] = fmaf(g[j], c[j][e], du[e]);
        const uint2 inf = rec_entry<G::L>(gm, i0, info, 1 + j, active);
        const int32_t y = rec_entry<G::L>(gm, r0, rec, 1 + j, active);
        if (active) {
            if (inf.x & kSingleBit) {
                const float decay = 1.0f * etalam;
                float x[G::E];
#pragma unroll
                for (int e = 0; e < G::E; ++e) x[e] = fmaf(-decay, c[j][e], c[j][e]) + g[j] * xu[e];
                store_row<D, DT>(p.C, y, lig, x, p.seed, t0, ctx_table);
            } else {
                float4* dst = reinterpret_cast<float4*>(p.slab + (int64_t)inf.x * D + lig * G::E);
#pragma unroll
                for (int q = 0; q < G::E / 4; ++q)
                    st_cg(dst + q, make_float4(g[j] * xu[4 * q], g[j] * xu[4 * q + 1], g[j] * xu[4 * q + 2],
                                               g[j] * xu[4 * q + 3]));
            }
        }
    }
    const uint2 inf0 = shfl_w(gm, i0, 0, G::L);
    if (active) {
        if (inf0.x & kSingleBit) {
            const float decay = (float)(p.K + 1) * etalam;
#pragma unroll
            for (int e = 0; e < G::E; ++e) xu[e] = fmaf(-decay, xu[e], xu[e]) + du[e];
            store_row<D, DT>(p.U, u, lig, xu, p.seed, t0, 0u);
        } else {
            float4* dst = reinterpret_cast<float4*>(p.slab + (int64_t)inf0.x * D + lig * G::E);
#pragma unroll
            for (int q = 0; q < G::E / 4; ++q) st_cg(dst + q, make_float4(du[4 * q], du[4 * q + 1], du[4 * q + 2], du[4 * q + 3]));
        }
    }
}

// Staged gather body (any K): the K+1 context rows are staged in shared
// memory (ctx_stage: (K+1) x 32 lanes x E floats), the dots reduced JB at a
// time.  Same arithmetic, in the same order, as the register body.
template <int D, int DT>
__device__ __forceinline__ void sample_body_staged(const DataParams& p, int lig, int lane, bool active, float eta,
                                                   uint64_t t0, uint32_t gm, int32_t r0, uint2 i0, const int32_t* rec,
                                                   const uint2* info, float* ctx_stage) {
    using G = Geom<D, DT>;
    constexpr int CH = G::E <= 4 ? 8 : 4;  // context rows in flight per lane
    const int32_t u = __shfl_sync(gm, r0, 0, G::L);
    float xu[G::E];
    load_row<D, DT>(p.U, u, lig, xu);
    for (int j0 = 0; j0 <= p.K; j0 += CH) {
        float c[CH][G::E];
#pragma unroll
        for (int jj = 0; jj < CH; ++jj) {
            const int j = j0 + jj;
            int32_t y = rec_entry<G::L>(gm, r0, rec, 1 + j, active && j <= p.K);
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
    const uint32_t ctx_table = p.order == 2 ? 1u : 0u;
    const float etalam = eta * p.lambda;
    float du[G::E];
#pragma unroll
    for (int e = 0; e < G::E; ++e) du[e] = 0.0f;
    constexpr int JB = 8;  // dot products reduced together (independent shuffles)
    for (int j0 = 0; j0 <= p.K; j0 += JB) {
        float sj[JB];
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
            sj[jj] = 0.0f;
            if (j0 + jj <= p.K) {
                const float4* ld = reinterpret_cast<const float4*>(ctx_stage + ((j0 + jj) * 32 + lane) * G::E);
#pragma unroll
                for (int q = 0; q < G::E / 4; ++q) {
                    const float4 a = ld[q];
                    sj[jj] = fmaf(xu[4 * q], a.x, sj[jj]);
                    sj[jj] = fmaf(xu[4 * q + 1], a.y, sj[jj]);
                    sj[jj] = fmaf(xu[4 * q + 2], a.z, sj[jj]);
                    sj[jj] = fmaf(xu[4 * q + 3], a.w, sj[jj]);
                }
            }
        }
#pragma unroll
        for (int o = G::L / 2; o >= 1; o >>= 1)
#pragma unroll
            for (int jj = 0; jj < JB; ++jj) sj[jj] += __shfl_xor_sync(0xFFFFFFFFu, sj[jj], o);
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
            const int j = j0 + jj;
            if (j > p.K) break;
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
            const float sig = 1.0f / (1.0f + expf(-sj[jj]));
            const float g = j == 0 ? eta * (1.0f - sig) : -eta * p.alpha_neg * sig;
#pragma unroll
            for (int e = 0; e < G::E; ++e) du[e] = fmaf(g, c[e], du[e]);
            const uint2 inf = rec_entry<G::L>(gm, i0, info, 1 + j, active);
            const int32_t y = rec_entry<G::L>(gm, r0, rec, 1 + j, active);
            if (active) {
                if (inf.x & kSingleBit) {
                    // the only reader of row y in this batch: write it now
                    const float decay = 1.0f * etalam;
                    float x[G::E];
#pragma unroll
                    for (int e = 0; e < G::E; ++e) x[e] = fmaf(-decay, c[e], c[e]) + g * xu[e];
                    store_row<D, DT>(p.C, y, lig, x, p.seed, t0, ctx_table);
                } else {
                    float4* dst = reinterpret_cast<float4*>(p.slab + (int64_t)inf.x * D + lig * G::E);
#pragma unroll
                    for (int q = 0; q < G::E / 4; ++q)
                        st_cg(dst + q, make_float4(g * xu[4 * q], g * xu[4 * q + 1], g * xu[4 * q + 2], g * xu[4 * q + 3]));
                }
            }
        }
    }
    const uint2 inf0 = shfl_w(gm, i0, 0, G::L);
    if (active) {
        if (inf0.x & kSingleBit) {
            const float decay = (float)(p.K + 1) * etalam;
#pragma unroll
            for (int e = 0; e < G::E; ++e) xu[e] = fmaf(-decay, xu[e], xu[e]) + du[e];
            store_row<D, DT>(p.U, u, lig, xu, p.seed, t0, 0u);
        } else {
            float4* dst = reinterpret_cast<float4*>(p.slab + (int64_t)inf0.x * D + lig * G::E);
#pragma unroll
            for (int q = 0; q < G::E / 4; ++q) st_cg(dst + q, make_float4(du[4 * q], du[4 * q + 1], du[4 * q + 2], du[4 * q + 3]));
        }
    }
}

template <int D, int DT, bool PDL = false>
__device__ __forceinline__ void sample_item(const DataParams& p, int64_t s_local, int lig, int lane, bool active,
                                            float eta, uint64_t t0, float* ctx_stage) {
    using G = Geom<D, DT>;
    const int R = p.K + 2;
    const int64_t sbase = (active ? s_local : 0) * R;
    const int32_t* rec = p.rec + sbase;
    const uint2* info = p.slot_info + sbase;
    const uint32_t gm = group_mask<G::L>(lane / G::L);
    const int32_t r0 = (active && lig < R) ? rec[lig] : 0;
    const uint2 i0 = (active && lig < R) ? info[lig] : make_uint2(0u, 0u);
    if constexpr (PDL) pdl_wait();  // the tables' rows: written by the previous kernel
    if constexpr (G::E <= 4) {
        if (p.K < 6) {
            sample_body_reg<D, DT, 6>(p, lig, active, eta, t0, gm, r0, i0, rec, info);
            return;
        }
        if (p.K < 8) {
            sample_body_reg<D, DT, 8>(p, lig, active, eta, t0, gm, r0, i0, rec, info);
            return;
        }
    }
    sample_body_staged<D, DT>(p, lig, lane, active, eta, t0, gm, r0, i0, rec, info, ctx_stage);
}

// ---------------------------------------------------------------------------
// Per shared segment: fixed-order sum of its contiguous slab entries and the
// write-back.
// ---------------------------------------------------------------------------
template <int D, int DT>
__device__ __forceinline__ void segment_item(const DataParams& p, uint4 d, int lig, bool active, float eta,
                                             uint64_t t0) {
    using G = Geom<D, DT>;
    constexpr int PF = G::E <= 4 ? 8 : 4;  // slab entries in flight per lane
    if (!active) return;
    // d = {first position, length | long bit, row, pair count}
    const uint32_t len = d.y & ~kLongBit;
    const uint32_t rowid = d.z & ((1u << p.row_bits) - 1u);
    const bool is_c = p.order == 2 && rowid >= (uint32_t)p.n_nodes;
    void* table = is_c ? p.C : p.U;
    const int64_t row = is_c ? (int64_t)rowid - p.n_nodes : (int64_t)rowid;
    float x[G::E];
    load_row<D, DT>(table, row, lig, x);
    float acc[G::E];
#pragma unroll
    for (int e = 0; e < G::E; ++e) acc[e] = 0.0f;
    const float* base = p.slab + (int64_t)d.x * D + lig * G::E;
    for (uint32_t c0 = 0; c0 < len; c0 += kChunk) {
        float part[G::E];
#pragma unroll
        for (int e = 0; e < G::E; ++e) part[e] = 0.0f;
#pragma unroll
        for (uint32_t k0 = 0; k0 < kChunk; k0 += PF) {
            float4 buf[PF][G::E / 4];
#pragma unroll
            for (int kk = 0; kk < PF; ++kk) {
                if (c0 + k0 + kk < len) {
                    const float4* src = reinterpret_cast<const float4*>(base + (int64_t)(c0 + k0 + kk) * D);
#pragma unroll
                    for (int q = 0; q < G::E / 4; ++q) buf[kk][q] = ld_cg(src + q);
                }
            }
#pragma unroll
            for (int kk = 0; kk < PF; ++kk) {
                if (c0 + k0 + kk < len) {
#pragma unroll
                    for (int q = 0; q < G::E / 4; ++q) {
                        part[4 * q] += buf[kk][q].x;
                        part[4 * q + 1] += buf[kk][q].y;
                        part[4 * q + 2] += buf[kk][q].z;
                        part[4 * q + 3] += buf[kk][q].w;
                    }
                }
            }
        }
#pragma unroll
        for (int e = 0; e < G::E; ++e) acc[e] += part[e];
    }
    const float decay = (float)d.w * (eta * p.lambda);
#pragma unroll
    for (int e = 0; e < G::E; ++e) x[e] = fmaf(-decay, x[e], x[e]) + acc[e];
    store_row<D, DT>(table, row, lig, x, p.seed, t0, is_c ? 1u : 0u);
}

// Warps of an apply block: 16 when one order trains alone (a hub row's
// chunks are summed in fewer rounds), 8 when two orders train concurrently
// (smaller blocks interleave better with the other order's kernels).
constexpr int kApplyWarpsAlone = 16, kApplyWarpsShared = 8;

// A long shared segment summed by the NW warps of a CTA: warp w sums chunks
// w, w+NW, ... (entry order within a chunk); warp 0 adds the chunk partials
// in chunk order - the same order as segment_item, so the result does not
// depend on the number of warps.  Uses lane group 0 of each warp.  part:
// shared, NW x D floats.
template <int D, int DT, int NW>
__device__ __forceinline__ void long_segment_cta(const DataParams& p, uint4 d, float eta, uint64_t t0, float* part) {
    using G = Geom<D, DT>;
    constexpr int PF = G::E <= 4 ? 8 : 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool mine = lane < G::L;  // group 0 of the warp
    const int lig = lane;
    const uint32_t len = d.y & ~kLongBit;
    const uint32_t n_chunks = (len + kChunk - 1) / kChunk;
    const uint32_t rowid = d.z & ((1u << p.row_bits) - 1u);
    const bool is_c = p.order == 2 && rowid >= (uint32_t)p.n_nodes;
    void* table = is_c ? p.C : p.U;
    const int64_t row = is_c ? (int64_t)rowid - p.n_nodes : (int64_t)rowid;
    float x[G::E];
    if (warp == 0 && mine) load_row<D, DT>(table, row, lig, x);  // in flight during the sums
    float acc[G::E];
#pragma unroll
    for (int e = 0; e < G::E; ++e) acc[e] = 0.0f;
    const float* base = p.slab + (int64_t)d.x * D + (mine ? lig : 0) * G::E;
    for (uint32_t r0 = 0; r0 < n_chunks; r0 += NW) {
        const uint32_t c = r0 + (uint32_t)warp;
        if (mine && c < n_chunks) {
            float pt[G::E];
#pragma unroll
            for (int e = 0; e < G::E; ++e) pt[e] = 0.0f;
            const uint32_t c0 = c * kChunk;
#pragma unroll
            for (uint32_t k0 = 0; k0 < kChunk; k0 += PF) {
                float4 buf[PF][G::E / 4];
#pragma unroll
                for (int kk = 0; kk < PF; ++kk) {
                    if (c0 + k0 + kk < len) {
                        const float4* src = reinterpret_cast<const float4*>(base + (int64_t)(c0 + k0 + kk) * D);
#pragma unroll
                        for (int q = 0; q < G::E / 4; ++q) buf[kk][q] = ld_cg(src + q);
                    }
                }
#pragma unroll
                for (int kk = 0; kk < PF; ++kk) {
                    if (c0 + k0 + kk < len) {
#pragma unroll
                        for (int q = 0; q < G::E / 4; ++q) {
                            pt[4 * q] += buf[kk][q].x;
                            pt[4 * q + 1] += buf[kk][q].y;
                            pt[4 * q + 2] += buf[kk][q].z;
                            pt[4 * q + 3] += buf[kk][q].w;
                        }
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < G::E; ++e) part[warp * D + lig * G::E + e] = pt[e];
        }
        __syncthreads();
        if (warp == 0 && mine) {
            const uint32_t nr = min((uint32_t)NW, n_chunks - r0);
            for (uint32_t w = 0; w < nr; ++w)
#pragma unroll
                for (int e = 0; e < G::E; ++e) acc[e] += part[w * D + lig * G::E + e];
        }
        __syncthreads();
    }
    if (warp == 0 && mine) {
        const float decay = (float)d.w * (eta * p.lambda);
#pragma unroll
        for (int e = 0; e < G::E; ++e) x[e] = fmaf(-decay, x[e], x[e]) + acc[e];
        store_row<D, DT>(table, row, lig, x, p.seed, t0, is_c ? 1u : 0u);
    }
}

// ---------------------------------------------------------------------------
// Batched schedule: one launch per phase per batch.
// ---------------------------------------------------------------------------
constexpr size_t kMaxSmem = 200 * 1024;

// Gathers run in blocks of at most 4 warps at 8 blocks per SM (at most 64
// registers), so that a 4,096-sample batch (4,096 warps at d = 128) is
// resident in one wave and still leaves registers on every SM for the
// pre-pass kernels of the next chunk (one batch at 72 registers filled 95%
// of the register file, and any pre-pass block displaced gather warps).
constexpr int kGatherWarps = 4;

template <int D, int DT, bool PDL>
__global__ void __launch_bounds__(kGatherWarps * 32, 8) k_gather(DataParams p, int b) {
    using G = Geom<D, DT>;
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    if constexpr (PDL) pdl_launch_dependents();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G::L, lig = lane % G::L;
    const int64_t s_begin = (int64_t)b * p.batch;
    const int64_t s_end = min(s_begin + p.batch, p.chunk_samples);
    const int64_t s_local = s_begin + ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * G::GPW + grp;
    float* stage = smem + (size_t)warp * (p.K + 1) * 32 * G::E;
    const uint64_t tc = p.t_chunk_dev ? *p.t_chunk_dev : p.t_chunk;
    sample_item<D, DT, PDL>(p, s_local, lig, lane, s_local < s_end, p.eta[b], tc + (uint64_t)s_begin, stage);
}

// Blocks [0, g_long) take the batch's long shared segments, one per CTA; the
// other blocks take the short ones, one per lane group.

template <int D, int DT, int NW>
__global__ void __launch_bounds__(NW * 32) k_apply(DataParams p, int b, int g_long) {
    using G = Geom<D, DT>;
    __shared__ float part[NW * D];
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G::L, lig = lane % G::L;
    const uint32_t n_m = p.mcount[b];
    const uint32_t n_long = p.lcount[b];
    const uint4* md = p.mdesc + (size_t)b * p.mcap;
    const uint64_t t0 = (p.t_chunk_dev ? *p.t_chunk_dev : p.t_chunk) + (uint64_t)b * (uint64_t)p.batch;
    const float eta = p.eta[b];
    if ((int)blockIdx.x < g_long) {
        // descriptors come from the pre-pass: read before the wait
        uint4 d = blockIdx.x < n_long ? p.ldesc[(size_t)b * p.lcap + blockIdx.x] : make_uint4(0u, 0u, 0u, 0u);
        pdl_wait();  // the slab and the rows: written by the gather
        for (uint32_t l = blockIdx.x; l < n_long; l += (uint32_t)g_long) {
            if (l != blockIdx.x) d = p.ldesc[(size_t)b * p.lcap + l];
            long_segment_cta<D, DT, NW>(p, d, eta, t0, part);
        }
        return;
    }
    const int64_t groups = (int64_t)(gridDim.x - g_long) * (blockDim.x >> 5) * G::GPW;
    const int64_t m0 = ((int64_t)(blockIdx.x - g_long) * (blockDim.x >> 5) + warp) * G::GPW + grp;
    uint4 d = m0 < n_m ? md[m0] : make_uint4(0u, 0u, 0u, 0u);
    pdl_wait();  // the slab and the rows: written by the gather
    for (int64_t m = m0; m < n_m; m += groups) {
        if (m != m0) d = md[m];
        if (d.y & kLongBit) continue;
        segment_item<D, DT>(p, d, lig, true, eta, t0);
    }
}

// ---------------------------------------------------------------------------
// Persistent schedule (LINE_MODE_PERSISTENT): one cooperative launch per
// chunk; one CTA of W warps per SM stays resident for all the chunk's
// batches.  For batch b:
//   gather  warp u takes the samples of units u, u + NW, ... (NW warps in
//           all; a unit is one sample per lane group).  A sample's K+2 rows
//           (U[u], then the context rows) are brought into the warp's
//           shared-memory slot by bulk copies (cp.async.bulk) that complete
//           on the slot's mbarrier; with two slots the next unit's copies run
//           while one unit is computed.  The arithmetic is the batched
//           gather's, reading the rows from shared memory; singleton rows
//           are written back, shared rows' contributions go to the slab.
//   barrier (grid-wide)
//   apply   each warp first starts the copies of its first unit of batch b+1
//           for the rows that batch b does not touch (b's row map: those rows
//           are not written in batch b); then every CTA applies some of
//           batch b's long shared segments (all its warps on one segment)
//           and every lane group some of its short ones.
//   barrier
// The rows of batch b+1 that batch b touches are copied after the second
// barrier.  Every wait is bounded: a barrier or a copy that does not finish
// within spin_limit polls records DEV_ERR_TIMEOUT, raises the abort word,
// waits (bounded) for the warp's own copies in flight, and returns.
// ---------------------------------------------------------------------------
constexpr int kPersistMaxWarps = 16;
constexpr int kPersistDefaultWarps = 16;

__device__ __forceinline__ void fail_abort(const DataParams& p) {
    atomicOr(p.status, DEV_ERR_TIMEOUT);
    atomicExch(p.abort_word, 1u);
}

// Grid-wide barrier: round r completes when all CTAs have arrived r+1 times
// (gbar[0] counts arrivals; the last arriver publishes r+1 in gbar[1]).
// Every thread's earlier global writes are visible to every CTA after it.
// Returns false when the wait ran out or another CTA aborted.
__device__ __forceinline__ bool grid_barrier(const DataParams& p, uint32_t r, uint32_t* s_flag) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = true;
        const uint32_t old = atom_add_acq_rel(p.gbar, 1u);
        if (old == (r + 1u) * gridDim.x - 1u) {
            st_release(p.gbar + 1, r + 1u);
        } else {
            int64_t it = 0;
            while (ld_acquire(p.gbar + 1) < r + 1u) {
                if (++it > p.spin_limit || *(volatile const uint32_t*)p.abort_word) {
                    ok = false;
                    break;
                }
                if (it > 64) __nanosleep(32);
            }
        }
        if (!ok) fail_abort(p);
        *s_flag = ok ? 1u : 0u;
    }
    __syncthreads();
    return *s_flag != 0u;
}

// One lane group's sample from its staged rows (slot: row 0 = U[u], rows
// 1..K+1 = the context rows, D values each in the table's type).  The
// arithmetic is sample_body_staged's, in the same order.
template <int D, int DT>
__device__ __forceinline__ void slot_row(const unsigned char* set, int j, int lig, float (&v)[Geom<D, DT>::E]) {
    using G = Geom<D, DT>;
    if constexpr (DT == LINE_DTYPE_F32) {
        const float4* q = reinterpret_cast<const float4*>(set + (size_t)j * D * 4 + (size_t)lig * G::E * 4);
#pragma unroll
        for (int k = 0; k < G::NV; ++k) {
            const float4 a = q[k];
            v[4 * k] = a.x;
            v[4 * k + 1] = a.y;
            v[4 * k + 2] = a.z;
            v[4 * k + 3] = a.w;
        }
    } else {
        const uint2* q = reinterpret_cast<const uint2*>(set + (size_t)j * D * 2 + (size_t)lig * G::E * 2);
#pragma unroll
        for (int k = 0; k < G::NV; ++k) {
            const uint2 a = q[k];
            v[4 * k] = __uint_as_float(a.x << 16);
            v[4 * k + 1] = __uint_as_float(a.x & 0xFFFF0000u);
            v[4 * k + 2] = __uint_as_float(a.y << 16);
            v[4 * k + 3] = __uint_as_float(a.y & 0xFFFF0000u);
        }
    }
}

template <int D, int DT>
__device__ __forceinline__ void sample_body_slot(const DataParams& p, int lig, bool active, float eta, uint64_t t0,
                                                 uint32_t gm, int32_t r0, uint2 i0, const int32_t* rec,
                                                 const uint2* info, const unsigned char* set) {
    using G = Geom<D, DT>;
    constexpr int JB = 8;
    const int32_t u = __shfl_sync(gm, r0, 0, G::L);
    float xu[G::E];
    slot_row<D, DT>(set, 0, lig, xu);
    const uint32_t ctx_table = p.order == 2 ? 1u : 0u;
    const float etalam = eta * p.lambda;
    float du[G::E];
#pragma unroll
    for (int e = 0; e < G::E; ++e) du[e] = 0.0f;
    for (int j0 = 0; j0 <= p.K; j0 += JB) {
        float sj[JB];
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
            sj[jj] = 0.0f;
            if (j0 + jj <= p.K) {
                float c[G::E];
                slot_row<D, DT>(set, 1 + j0 + jj, lig, c);
#pragma unroll
                for (int e = 0; e < G::E; ++e) sj[jj] = fmaf(xu[e], c[e], sj[jj]);
            }
        }
#pragma unroll
        for (int o = G::L / 2; o >= 1; o >>= 1)
#pragma unroll
            for (int jj = 0; jj < JB; ++jj) sj[jj] += __shfl_xor_sync(0xFFFFFFFFu, sj[jj], o);
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
            const int j = j0 + jj;
            if (j > p.K) break;
            float c[G::E];
            slot_row<D, DT>(set, 1 + j, lig, c);
            const float sig = 1.0f / (1.0f + expf(-sj[jj]));
            const float g = j == 0 ? eta * (1.0f - sig) : -eta * p.alpha_neg * sig;
#pragma unroll
            for (int e = 0; e < G::E; ++e) du[e] = fmaf(g, c[e], du[e]);
            const uint2 inf = rec_entry<G::L>(gm, i0, info, 1 + j, active);
            const int32_t y = rec_entry<G::L>(gm, r0, rec, 1 + j, active);
            if (active) {
                if (inf.x & kSingleBit) {
                    const float decay = 1.0f * etalam;
                    float x[G::E];
#pragma unroll
                    for (int e = 0; e < G::E; ++e) x[e] = fmaf(-decay, c[e], c[e]) + g * xu[e];
                    store_row<D, DT>(p.C, y, lig, x, p.seed, t0, ctx_table);
                } else {
                    float4* dst = reinterpret_cast<float4*>(p.slab + (int64_t)inf.x * D + lig * G::E);
#pragma unroll
                    for (int q = 0; q < G::E / 4; ++q)
                        st_cg(dst + q, make_float4(g * xu[4 * q], g * xu[4 * q + 1], g * xu[4 * q + 2], g * xu[4 * q + 3]));
                }
            }
        }
    }
    const uint2 inf0 = shfl_w(gm, i0, 0, G::L);
    if (active) {
        if (inf0.x & kSingleBit) {
            const float decay = (float)(p.K + 1) * etalam;
#pragma unroll
            for (int e = 0; e < G::E; ++e) xu[e] = fmaf(-decay, xu[e], xu[e]) + du[e];
            store_row<D, DT>(p.U, u, lig, xu, p.seed, t0, 0u);
        } else {
            float4* dst = reinterpret_cast<float4*>(p.slab + (int64_t)inf0.x * D + lig * G::E);
#pragma unroll
            for (int q = 0; q < G::E / 4; ++q) st_cg(dst + q, make_float4(du[4 * q], du[4 * q + 1], du[4 * q + 2], du[4 * q + 3]));
        }
    }
}

// Starts the bulk copies of rows j (bit j of `want`, j < K+2) of a lane
// group's sample into its row set, completing on `bar`.  arrive: this is the
// group's last issue for the slot's current phase (an arrival, with the
// bytes); otherwise only the bytes are announced.  Row j of the sample is
// U[rec[0]] for j = 0, Ctx[rec[j]] otherwise.
template <int D, int DT>
__device__ __forceinline__ void issue_rows(const DataParams& p, const int32_t* rec, int lig, uint32_t gm, int R,
                                           uint64_t want, bool arrive, unsigned char* set, uint64_t* bar) {
    using G = Geom<D, DT>;
    constexpr uint32_t kRowBytes = D * (DT == LINE_DTYPE_F32 ? 4 : 2);
    const uint32_t bytes = (uint32_t)__popcll(want) * kRowBytes;
    if (lig == 0) {
        if (arrive) mbar_arrive_expect_tx(bar, bytes);
        else if (bytes) mbar_expect_tx(bar, bytes);
    }
    __syncwarp(gm);
    for (int j = lig; j < R; j += G::L) {
        if ((want >> j) & 1ull) {
            const int32_t row = rec[j];
            const void* table = j == 0 ? p.U : p.C;
            const unsigned char* src = reinterpret_cast<const unsigned char*>(table) + (size_t)row * kRowBytes;
            bulk_load(set + (size_t)j * kRowBytes, src, kRowBytes, bar);
        }
    }
}

// A long shared segment summed by all W warps of the CTA (runtime W): warp w
// sums chunks w, w+W, ... (entry order within a chunk); warp 0 adds the
// chunk partials in chunk order, as segment_item does.  part: W x D floats.
template <int D, int DT>
__device__ __forceinline__ void long_segment_rt(const DataParams& p, uint4 d, float eta, uint64_t t0, float* part, int W) {
    using G = Geom<D, DT>;
    constexpr int PF = G::E <= 4 ? 8 : 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool mine = lane < G::L;
    const int lig = lane;
    const uint32_t len = d.y & ~kLongBit;
    const uint32_t n_chunks = (len + kChunk - 1) / kChunk;
    const uint32_t rowid = d.z & ((1u << p.row_bits) - 1u);
    const bool is_c = p.order == 2 && rowid >= (uint32_t)p.n_nodes;
    void* table = is_c ? p.C : p.U;
    const int64_t row = is_c ? (int64_t)rowid - p.n_nodes : (int64_t)rowid;
    float x[G::E];
    if (warp == 0 && mine) load_row<D, DT>(table, row, lig, x);
    float acc[G::E];
#pragma unroll
    for (int e = 0; e < G::E; ++e) acc[e] = 0.0f;
    const float* base = p.slab + (int64_t)d.x * D + (mine ? lig : 0) * G::E;
    for (uint32_t r0 = 0; r0 < n_chunks; r0 += (uint32_t)W) {
        const uint32_t c = r0 + (uint32_t)warp;
        if (mine && c < n_chunks) {
            float pt[G::E];
#pragma unroll
            for (int e = 0; e < G::E; ++e) pt[e] = 0.0f;
            const uint32_t c0 = c * kChunk;
#pragma unroll
            for (uint32_t k0 = 0; k0 < kChunk; k0 += PF) {
                float4 buf[PF][G::E / 4];
#pragma unroll
                for (int kk = 0; kk < PF; ++kk)
                    if (c0 + k0 + kk < len)
#pragma unroll
                        for (int q = 0; q < G::E / 4; ++q)
                            buf[kk][q] = ld_cg(reinterpret_cast<const float4*>(base + (int64_t)(c0 + k0 + kk) * D) + q);
#pragma unroll
                for (int kk = 0; kk < PF; ++kk)
                    if (c0 + k0 + kk < len)
#pragma unroll
                        for (int q = 0; q < G::E / 4; ++q) {
                            pt[4 * q] += buf[kk][q].x;
                            pt[4 * q + 1] += buf[kk][q].y;
                            pt[4 * q + 2] += buf[kk][q].z;
                            pt[4 * q + 3] += buf[kk][q].w;
                        }
            }
#pragma unroll
            for (int e = 0; e < G::E; ++e) part[warp * D + lig * G::E + e] = pt[e];
        }
        __syncthreads();
        if (warp == 0 && mine) {
            const uint32_t nr = min((uint32_t)W, n_chunks - r0);
            for (uint32_t w = 0; w < nr; ++w)
#pragma unroll
                for (int e = 0; e < G::E; ++e) acc[e] += part[w * D + lig * G::E + e];
        }
        __syncthreads();
    }
    if (warp == 0 && mine) {
        const float decay = (float)d.w * (eta * p.lambda);
#pragma unroll
        for (int e = 0; e < G::E; ++e) x[e] = fmaf(-decay, x[e], x[e]) + acc[e];
        store_row<D, DT>(table, row, lig, x, p.seed, t0, is_c ? 1u : 0u);
    }
}

// Row bytes of one lane group's sample set, rounded up to 128.
__host__ __device__ inline size_t persist_set_bytes(int dim, int dtype, int K) {
    return (((size_t)(K + 2) * dim * (dtype == LINE_DTYPE_F32 ? 4 : 2)) + 127) & ~(size_t)127;
}

// Dynamic shared memory of a W-warp CTA: the warps' row slots, the long
// segments' partials (W x D floats) and two mbarriers per warp.
__host__ __device__ inline size_t persist_smem_bytes(int dim, int dtype, int K, int W, int slots, int gpw) {
    return (size_t)W * slots * gpw * persist_set_bytes(dim, dtype, K) + (size_t)W * dim * sizeof(float) +
           (size_t)W * 2 * sizeof(uint64_t);
}

template <int D, int DT>
__global__ void __launch_bounds__(kPersistMaxWarps * 32, 1) k_persistent(DataParams p) {
    using G = Geom<D, DT>;
    extern __shared__ __align__(128) unsigned char psm[];
    __shared__ uint32_t s_flag;
    const int W = (int)(blockDim.x >> 5);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G::L, lig = lane % G::L;
    const uint32_t gm = group_mask<G::L>(grp);
    const int R = p.K + 2;
    const size_t set_bytes = persist_set_bytes(D, DT, p.K);
    const int slots = p.slots;
    unsigned char* wslots = psm + (size_t)warp * slots * G::GPW * set_bytes;
    float* part = reinterpret_cast<float*>(psm + (size_t)W * slots * G::GPW * set_bytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(part + (size_t)W * D) + 2 * warp;
    if (lane == 0) {
        mbar_init(bars, G::GPW);  // one arrival per lane group and phase
        mbar_init(bars + 1, G::GPW);
        mbar_init_fence();
    }
    __syncwarp();
    const int64_t NW = (int64_t)gridDim.x * W;                 // warps in all
    const int64_t uwarp = (int64_t)blockIdx.x * W + warp;      // this warp
    uint32_t par0 = 0, par1 = 0;                               // phase parity of each slot
    bool pending0 = false, pending1 = false;                   // copies issued, not yet waited for
    uint64_t pre_want = 0;                                     // rows of unit 0 already requested (prefetch)
    bool prefetched = false;
    uint32_t round = 0;
    bool ok = true;
    const uint64_t all_rows = R >= 64 ? ~0ull : ((1ull << R) - 1ull);
    for (int b = 0; b < p.n_batches && ok; ++b) {
        const int64_t s_begin = (int64_t)b * p.batch;
        const int64_t nb = min((int64_t)p.batch, p.chunk_samples - s_begin);
        const int64_t units = (nb + G::GPW - 1) / G::GPW;
        const uint64_t t0 = p.t_chunk + (uint64_t)s_begin;
        const float eta = p.eta[b];
        const int64_t n_mine = uwarp < units ? (units - 1 - uwarp) / NW + 1 : 0;
        // ---- gather of batch b
        // copies of the first two units (unit 0's prefetched rows are in flight)
        for (int k = 0; k < 2 && k < n_mine; ++k) {
            const int64_t s_local = s_begin + (uwarp + k * NW) * G::GPW + grp;
            const bool active = s_local < s_begin + nb;
            const int32_t* rec = p.rec + (active ? s_local : 0) * R;
            uint64_t want = active ? all_rows : 0ull;
            if (k == 0 && prefetched) want &= ~pre_want;
            fence_proxy_async_global();
            issue_rows<D, DT>(p, rec, lig, gm, R, want, true, wslots + (size_t)k * G::GPW * set_bytes + grp * set_bytes,
                              bars + k);
            if (k == 0) pending0 = true;
            else pending1 = true;
        }
        prefetched = false;
        for (int64_t k = 0; k < n_mine && ok; ++k) {
            const int sl = (int)(k & 1);
            const int64_t s_local = s_begin + (uwarp + k * NW) * G::GPW + grp;
            const bool active = s_local < s_begin + nb;
            // wait for the unit's rows
            uint64_t* bar = bars + sl;
            const uint32_t par = sl ? par1 : par0;
            int64_t it = 0;
            while (!mbar_try_wait(bar, par)) {
                if (++it > p.spin_limit || *(volatile const uint32_t*)p.abort_word) {
                    ok = false;
                    break;
                }
            }
            ok = __all_sync(0xFFFFFFFFu, ok);
            if (!ok) break;
            if (sl) {
                par1 ^= 1u;
                pending1 = false;
            } else {
                par0 ^= 1u;
                pending0 = false;
            }
            const unsigned char* set = wslots + (size_t)sl * G::GPW * set_bytes + grp * set_bytes;
            const int64_t sbase = (active ? s_local : 0) * R;
            const int32_t* rec = p.rec + sbase;
            const uint2* info = p.slot_info + sbase;
            const int32_t r0 = (active && lig < R) ? rec[lig] : 0;
            const uint2 i0 = (active && lig < R) ? info[lig] : make_uint2(0u, 0u);
            sample_body_slot<D, DT>(p, lig, active, eta, t0, gm, r0, i0, rec, info, set);
            // the slot's rows are read: it may be refilled by bulk copies
            fence_proxy_async_smem();
            __syncwarp();
            if (k + 2 < n_mine) {
                const int64_t s2 = s_begin + (uwarp + (k + 2) * NW) * G::GPW + grp;
                const bool act2 = s2 < s_begin + nb;
                issue_rows<D, DT>(p, p.rec + (act2 ? s2 : 0) * R, lig, gm, R, act2 ? all_rows : 0ull, true,
                                  wslots + (size_t)sl * G::GPW * set_bytes + grp * set_bytes, bar);
                if (sl) pending1 = true;
                else pending0 = true;
            }
        }
        if (!__all_sync(0xFFFFFFFFu, ok)) ok = false;
        if (!ok) {
            if (lane == 0) fail_abort(p);
            break;
        }
        if (!grid_barrier(p, round++, &s_flag)) {
            ok = false;
            break;
        }
        // ---- apply of batch b; first the prefetch of batch b+1's rows that
        // batch b does not touch
        if (b + 1 < p.n_batches) {
            const int64_t s1_begin = (int64_t)(b + 1) * p.batch;
            const int64_t nb1 = min((int64_t)p.batch, p.chunk_samples - s1_begin);
            const int64_t units1 = (nb1 + G::GPW - 1) / G::GPW;
            if (uwarp < units1) {
                const int64_t s_local = s1_begin + uwarp * G::GPW + grp;
                const bool active = s_local < s1_begin + nb1;
                const int32_t* rec = p.rec + (active ? s_local : 0) * R;
                // rows of the group's sample that batch b does not touch
                bool free_row = false;
                if (active && lig < R) {
                    const uint32_t rowid = (uint32_t)rec[lig] + (lig > 0 && p.order == 2 ? (uint32_t)p.n_nodes : 0u);
                    const uint32_t db = dep_bit(rowid);
                    free_row = !((__ldcg(p.depmap + (size_t)b * kDepWords + (db >> 5)) >> (db & 31u)) & 1u);
                }
                uint32_t fm = __ballot_sync(0xFFFFFFFFu, free_row);
                fm = G::L == 32 ? fm : (fm >> (grp * G::L)) & ((1u << G::L) - 1u);
                pre_want = (uint64_t)fm;  // rows >= L: copied after the barrier
                fence_proxy_async_global();
                issue_rows<D, DT>(p, rec, lig, gm, R, pre_want, false, wslots + grp * set_bytes, bars);
                prefetched = true;
                pending0 = true;
            }
        }
        {
            // long shared segments: one CTA each
            const uint32_t n_long = p.lcount[b];
            for (uint32_t l = blockIdx.x; l < n_long; l += gridDim.x)
                long_segment_rt<D, DT>(p, p.ldesc[(size_t)b * p.lcap + l], eta, t0, part, W);
            // short ones: one lane group each
            const uint32_t n_m = p.mcount[b];
            const uint4* md = p.mdesc + (size_t)b * p.mcap;
            for (int64_t m = uwarp * G::GPW + grp; m < n_m; m += NW * G::GPW) {
                const uint4 d = md[m];
                if (d.y & kLongBit) continue;
                segment_item<D, DT>(p, d, lig, true, eta, t0);
            }
        }
        if (!grid_barrier(p, round++, &s_flag)) {
            ok = false;
            break;
        }
    }
    if (!ok) {
        // wait (bounded) for this warp's copies still in flight, then return
        for (int sl = 0; sl < 2; ++sl) {
            if (!(sl ? pending1 : pending0)) continue;
            uint64_t* bar = bars + sl;
            const uint32_t par = sl ? par1 : par0;
            for (int64_t it = 0; it <= p.spin_limit && !mbar_try_wait(bar, par); ++it) {
            }
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
    int walk;  // 1: slots 0 and 1 come from the walk sampler (no arc draw here)
    int32_t* rec;
    uint64_t* items;  // null: records only (Hogwild schedule)
    uint64_t* t_out;  // receives t_chunk (read by graph replays of the data phase)
};

__device__ __forceinline__ uint64_t make_item(uint32_t rowid, uint32_t s_local, uint32_t slot) {
    return ((uint64_t)rowid << 32) | ((s_local << kSlotBits) | slot);
}

__global__ void k_chunk_draws(PrepassParams p) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && p.t_out) *p.t_out = p.t_chunk;
    const uint32_t C1 = (uint32_t)p.K + 1u, R = (uint32_t)p.K + 2u;
    const uint32_t total = (uint32_t)p.chunk_samples * C1;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const uint32_t s = q / C1;
        const uint32_t c = q - s * C1;
        const uint4 w = draw_words(p.seed, 0u, p.t_chunk + (uint64_t)s, c);
        const uint32_t ctx_off = p.order == 2 ? (uint32_t)p.n_nodes : 0u;
        const uint32_t base = s * R;
        if (c == 0) {
            if (p.walk) continue;
            const uint32_t e = alias_pick(p.edge_tab, (uint64_t)p.n_arcs, w);
            const int32_t u = __ldg(p.src + e), v = __ldg(p.dst + e);
            p.rec[base] = u;
            p.rec[base + 1] = v;
            if (p.items) {
                p.items[base] = make_item((uint32_t)u, s, 0u);
                p.items[base + 1] = make_item((uint32_t)v + ctx_off, s, 1u);
            }
        } else {
            const uint32_t y = alias_pick(p.neg_tab, (uint64_t)p.n_nodes, w);
            p.rec[base + 1 + c] = (int32_t)y;
            if (p.items) p.items[base + 1 + c] = make_item(y + ctx_off, s, 1u + c);
        }
    }
}

// ---------------------------------------------------------------------------
// Grouping of each batch's items by row.  Items of batch b occupy positions
// [b B (K+2), b B (K+2) + nb (K+2)) of the chunk, in (sample, slot) order.
// ---------------------------------------------------------------------------
constexpr int kBuckets = 256;            // bucket = 8-bit multiplicative hash of the row id

constexpr int kBucketThreads = 1024;
constexpr int kBucketWarps = kBucketThreads / 32;
constexpr uint32_t kPartItems = 16384;   // items of a batch per bucketing CTA
constexpr int kSortThreads = 256;        // one warp per bucket

struct GroupParams {
    int n_batches;
    int64_t batch;
    int64_t chunk_samples;
    uint32_t R, K, parts;  // parts: bucketing CTAs per batch
    uint32_t row_bits;
    const uint64_t* items;  // draws, (sample, slot) order
    uint64_t* bucketed;     // items grouped by bucket within each batch
    uint64_t* tmp;          // scratch of the same size
    uint32_t* gcnt;         // [n_batches][parts][256] bucket counts of each part
    uint32_t* boff;         // [n_batches][257] bucket starts within the batch
    // outputs
    uint2* slot_info;
    uint4* mdesc;
    uint32_t* mcount;
    uint32_t mcap;
    uint4* ldesc;
    uint32_t* lcount;
    uint32_t lcap;
    uint32_t* depmap;     // [n_batches][kDepWords] rows each batch touches (zeroed before), or null
};

__device__ __forceinline__ void batch_range(const GroupParams& q, int b, uint64_t* base, uint32_t* n) {
    const int64_t nb = min(q.batch, q.chunk_samples - (int64_t)b * q.batch);
    *base = (uint64_t)b * (uint64_t)q.batch * q.R;
    *n = (uint32_t)nb * q.R;
}

__global__ void __launch_bounds__(kBucketThreads) k_bucket_count(GroupParams q) {
    __shared__ uint32_t cnt[kBuckets];
    const int part = blockIdx.x, b = blockIdx.y;
    if (threadIdx.x < kBuckets) cnt[threadIdx.x] = 0;
    __syncthreads();
    uint64_t base;
    uint32_t n;
    batch_range(q, b, &base, &n);
    const uint32_t lo = min(n, (uint32_t)part * kPartItems), hi = min(n, lo + kPartItems);
    for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const uint32_t rowid = (uint32_t)(q.items[base + i] >> 32);
        atomicAdd(&cnt[bucket_of(rowid)], 1u);
        if (q.depmap) {
            const uint32_t db = dep_bit(rowid);
            atomicOr(q.depmap + (size_t)b * kDepWords + (db >> 5), 1u << (db & 31u));
        }
    }
    __syncthreads();
    if (threadIdx.x < kBuckets) q.gcnt[((size_t)b * q.parts + part) * kBuckets + threadIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one part: bucket start + the earlier parts' counts + the
// earlier warps' counts + the rank within the warp's rounds.
__global__ void __launch_bounds__(kBucketThreads) k_bucket_scatter(GroupParams q) {
    __shared__ uint32_t bstart[kBuckets], poff[kBuckets];
    __shared__ uint32_t wcnt[kBucketWarps][kBuckets];
    const int part = blockIdx.x, b = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t base;
    uint32_t n;
    batch_range(q, b, &base, &n);
    for (int i = threadIdx.x; i < kBucketWarps * kBuckets; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    if (threadIdx.x < kBuckets) {
        const uint32_t d = threadIdx.x;
        uint32_t tot = 0, before = 0;
        for (uint32_t pp = 0; pp < q.parts; ++pp) {
            const uint32_t c = q.gcnt[((size_t)b * q.parts + pp) * kBuckets + d];
            if (pp < (uint32_t)part) before += c;
            tot += c;
        }
        bstart[d] = tot;
        poff[d] = before;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int d = 0; d < kBuckets; ++d) {
            const uint32_t c = bstart[d];
            bstart[d] = run;
            run += c;
        }
    }
    __syncthreads();
    if (part == 0 && threadIdx.x <= kBuckets) q.boff[(size_t)b * (kBuckets + 1) + threadIdx.x] = threadIdx.x < kBuckets ? bstart[threadIdx.x] : n;
    const uint32_t lo = min(n, (uint32_t)part * kPartItems), hi = min(n, lo + kPartItems);
    const uint32_t per = (hi - lo + kBucketWarps - 1) / kBucketWarps;
    const uint32_t wlo = min(hi, lo + warp * per), whi = min(hi, wlo + per);
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t r = wlo; r < whi; r += 32) {
        const uint32_t i = r + lane;
        const bool valid = i < whi;
        const uint32_t d = valid ? bucket_of((uint32_t)(q.items[base + i] >> 32)) : 0xFFFFu;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        if (valid && (peers & lt) == 0) wcnt[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < kBuckets) {
        uint32_t run = 0;
        for (int w = 0; w < kBucketWarps; ++w) {
            const uint32_t c = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
    for (uint32_t r = wlo; r < whi; r += 32) {
        const uint32_t i = r + lane;
        const bool valid = i < whi;
        const uint64_t it = valid ? q.items[base + i] : 0ull;
        const uint32_t d = valid ? bucket_of((uint32_t)(it >> 32)) : 0xFFFFu;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t before = valid ? wcnt[warp][d] : 0u;
        if (valid) q.bucketed[base + bstart[d] + poff[d] + before + __popc(peers & lt)] = it;
        __syncwarp();
        if (valid && (peers & lt) == 0) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
}

// One stable 8-bit LSD pass of a warp over n items (global memory), by bits
// [shift, shift + 8) of the hashed row id.  cnt: the warp's 256 shared counters.
__device__ void warp_radix_pass(const uint64_t* src, uint64_t* dst, uint32_t n, uint32_t shift, uint32_t* cnt) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    for (int i = lane; i < kBuckets; i += 32) cnt[i] = 0;
    __syncwarp();
    for (uint32_t r = 0; r < n; r += 32) {
        const uint32_t i = r + lane;
        const bool valid = i < n;
        const uint32_t d = valid ? (hrow((uint32_t)(src[i] >> 32)) >> shift) & 255u : 0xFFFFu;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        if (valid && (peers & lt) == 0) cnt[d] += __popc(peers);
        __syncwarp();
    }
    // exclusive scan of the 256 counters: lane l owns counters 8l .. 8l+7
    uint32_t own = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) own += cnt[lane * 8 + k];
    uint32_t incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    uint32_t run = incl - own;
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t c = cnt[lane * 8 + k];
        cnt[lane * 8 + k] = run;
        run += c;
    }
    __syncwarp();
    for (uint32_t r = 0; r < n; r += 32) {
        const uint32_t i = r + lane;
        const bool valid = i < n;
        const uint64_t it = valid ? src[i] : 0ull;
        const uint32_t d = valid ? (hrow((uint32_t)(it >> 32)) >> shift) & 255u : 0xFFFFu;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t before = valid ? cnt[d] : 0u;
        if (valid) dst[before + __popc(peers & lt)] = it;
        __syncwarp();
        if (valid && (peers & lt) == 0) cnt[d] = before + __popc(peers);
        __syncwarp();
    }
}

constexpr uint32_t kWarpSortCap = 512;  // bucket sizes ranked directly in shared memory
constexpr int kSortBucketsPerCta = kSortThreads / 32;

// One warp per (bucket, batch): sort the bucket's items by row (stable), then
// find its segments.  Small buckets: a bitonic sort of (row, index) in shared
// memory; large ones: LSD radix passes in global memory.
__global__ void __launch_bounds__(kSortThreads) k_bucket_sort(GroupParams q) {
    extern __shared__ uint64_t sbuf[];  // per warp: 2 x kWarpSortCap items
    __shared__ uint32_t wcnt[kSortBucketsPerCta][kBuckets];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = blockIdx.x * kSortBucketsPerCta + warp, b = blockIdx.y;
    if (b >= q.n_batches || d >= kBuckets) return;
    uint64_t base;
    uint32_t n;
    batch_range(q, b, &base, &n);
    const uint32_t lo = q.boff[(size_t)b * (kBuckets + 1) + d], hi = q.boff[(size_t)b * (kBuckets + 1) + d + 1];
    const uint32_t c = hi - lo;
    if (c == 0) return;
    const uint64_t* a;
    if (c <= kWarpSortCap) {
        // bitonic sort of the unique keys (hrow(row) << 32 | index) over the
        // next power of two, padded with the largest key; then items by rank
        uint64_t* in = sbuf + (size_t)warp * 2 * kWarpSortCap;
        uint64_t* key = in + kWarpSortCap;
        uint32_t P = 32;
        while (P < c) P <<= 1;
        for (uint32_t i = lane; i < P; i += 32) {
            if (i < c) {
                const uint64_t it = q.bucketed[base + lo + i];
                in[i] = it;
                key[i] = ((uint64_t)hrow((uint32_t)(it >> 32)) << 32) | i;
            } else {
                key[i] = ~0ull;
            }
        }
        __syncwarp();
        for (uint32_t kk = 2; kk <= P; kk <<= 1) {
            for (uint32_t jj = kk >> 1; jj > 0; jj >>= 1) {
                for (uint32_t t = lane; t < P / 2; t += 32) {
                    const uint32_t i = ((t & ~(jj - 1)) << 1) | (t & (jj - 1));
                    const uint32_t l = i + jj;
                    const uint64_t x = key[i], y = key[l];
                    if ((x > y) == ((i & kk) == 0)) {
                        key[i] = y;
                        key[l] = x;
                    }
                }
                __syncwarp();
            }
        }
        // sorted items replace the keys in place (each lane reads, then writes, its own slots)
        for (uint32_t r = lane; r < c; r += 32) {
            const uint64_t it = in[(uint32_t)key[r]];
            key[r] = it;
        }
        __syncwarp();
        a = key;
    } else {  // a large bucket (a very skewed draw): radix passes over the hashed row
        uint64_t* x = q.bucketed + base + lo;
        uint64_t* y = q.tmp + base + lo;
        for (uint32_t sh = 0; sh < 32; sh += 8) {
            warp_radix_pass(x, y, c, sh, wcnt[warp]);
            uint64_t* t = x;
            x = y;
            y = t;
        }
        __syncwarp();
        a = x;
    }
    const uint32_t gpos = lo;  // position of the bucket's first item in the batch
    for (uint32_t i = lane; i < c; i += 32) {
        const uint32_t key = (uint32_t)(a[i] >> 32);
        if (i > 0 && (uint32_t)(a[i - 1] >> 32) == key) continue;
        uint32_t j = i + 1;
        while (j < c && (uint32_t)(a[j] >> 32) == key) ++j;
        const uint32_t len = j - i;
        const uint32_t head = (uint32_t)(gpos + i);
        uint32_t cnt = 0;
        for (uint32_t k = i; k < j; ++k) {
            const uint32_t v = (uint32_t)a[k];
            const uint32_t slot = v & kSlotMask;
            cnt += slot == 0 ? q.K + 1 : 1u;
            const uint32_t pos = (uint32_t)(gpos + k);
            q.slot_info[(v >> kSlotBits) * q.R + slot] = make_uint2(pos | (len == 1 ? kSingleBit : 0u), head);
        }
        if (len > 1) {
            uint32_t flagged = len;
            if (len > kChunk) {
                const uint32_t l = atomicAdd(q.lcount + b, 1u);
                q.ldesc[(size_t)b * q.lcap + l] = make_uint4(head, len, key, cnt);
                flagged |= kLongBit;
            }
            const uint32_t m = atomicAdd(q.mcount + b, 1u);
            q.mdesc[(size_t)b * q.mcap + m] = make_uint4(head, flagged, key, cnt);
        }
    }
}

// ---- Grouping of a batch by one thread-block cluster (batches of up to 8 x
// 3,584 items).  The items are split into P = 2^log_parts parts by the top
// bits of hrow(row) (a part is a contiguous range of buckets) and each part
// into 256 sub-buckets by the next 8 bits.  CTA rank r of batch b's cluster
// counts the (part, sub-bucket) sizes of the r-th slice of the batch's draws;
// after an exchange of counts every CTA knows where each of its keys
// (hrow(row) << 32 | index) goes in the owner's shared memory (distributed
// shared memory) and sends it there.  Each owner then sorts its sub-buckets
// (about 14 keys each: one thread; larger ones: one warp) and emits its
// segments.  The order, hence every position, is the same as the bucketed
// path's: (hrow(row), index).
constexpr int kGroupThreads = 512;
constexpr uint32_t kGroupCap = 4096;  // keys of a part held in shared memory
constexpr int kGroupMaxLog = 3;       // clusters of up to 8 CTAs (portable size)
constexpr int kSub = 256;             // sub-buckets of a part
constexpr int kGroupPerThread = 8;    // slice items per thread loaded at once

// In-place ascending sort of a[0 .. n) by one warp: a bitonic network whose
// comparators all put the minimum first (per merge size k the mirror
// comparator (i, k-1-i) within each k-block, then half-cleaners of strides
// k/4 .. 1); positions >= n act as +infinity, so comparators reaching past n
// are skipped.
__device__ __forceinline__ void warp_sort_keys(uint64_t* a, uint32_t n) {
    const int lane = threadIdx.x & 31;
    uint32_t N = 1;
    while (N < n) N <<= 1;
    for (uint32_t k = 2; k <= N; k <<= 1) {
        const uint32_t lh = 31 - __clz(k >> 1);
        for (uint32_t t = lane; t < N / 2; t += 32) {
            const uint32_t blk = t >> lh, off = t & ((k >> 1) - 1);
            const uint32_t i = blk * k + off, j = blk * k + k - 1 - off;
            if (j < n) {
                const uint64_t x = a[i], y = a[j];
                if (x > y) {
                    a[i] = y;
                    a[j] = x;
                }
            }
        }
        __syncwarp();
        for (uint32_t jj = k >> 2; jj > 0; jj >>= 1) {
            for (uint32_t t = lane; t < N / 2; t += 32) {
                const uint32_t i = ((t & ~(jj - 1)) << 1) | (t & (jj - 1)), j = i + jj;
                if (j < n) {
                    const uint64_t x = a[i], y = a[j];
                    if (x > y) {
                        a[i] = y;
                        a[j] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// The second half of the grouping of one part: sort its sub-buckets, write
// its bucket starts and emit its segments.  `a` holds the part's nq keys
// grouped by sub-bucket (s_start); inlined once for shared memory and once
// for the global scratch, so that the common case uses shared-memory accesses.
struct GroupShared {
    uint32_t* start;  // [kSub + 1] sub-bucket starts
    uint32_t* big;    // [kSub]
    uint32_t* nbig;
    uint32_t* mcnt;
    uint32_t* lcnt;
    uint32_t* mbase;
    uint32_t* lbase;
};

__device__ __forceinline__ void group_tail(const GroupParams& q, uint64_t* a, uint32_t nq, uint32_t n,
                                           uint32_t qbase, int b, uint32_t me, uint32_t P, int log_parts,
                                           const GroupShared& sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = kGroupThreads / 32;
    const uint32_t* s_start = sh.start;
    const uint32_t gpos = qbase;  // position of the part's first key in the batch
    // sort each sub-bucket by (hrow(row), index): up to 32 keys by ranks
    // within a warp, larger ones (a hot row) by a warp bitonic sort
    for (int sb = warp; sb < kSub; sb += kWarps) {
        const uint32_t s0 = s_start[sb], c = s_start[sb + 1] - s0;
        if (c <= 1) continue;
        if (c <= 32) {
            const uint64_t key = lane < (int)c ? a[s0 + lane] : ~0ull;
            uint32_t rank = 0;
            for (uint32_t l = 0; l < c; ++l) rank += __shfl_sync(0xFFFFFFFFu, key, l) < key;
            __syncwarp();
            if (lane < (int)c) a[s0 + rank] = key;
            __syncwarp();
        } else {
            warp_sort_keys(a + s0, c);
        }
    }
    __syncthreads();
    // bucket starts of the part's buckets: bucket (me, j) begins at
    // sub-bucket j << log_parts
    const uint32_t nbk = (uint32_t)kBuckets >> log_parts, d0 = me * nbk;
    for (uint32_t j = threadIdx.x; j < nbk; j += blockDim.x)
        q.boff[(size_t)b * (kBuckets + 1) + d0 + j] = qbase + s_start[j << log_parts];
    if (me == P - 1u && threadIdx.x == 0) q.boff[(size_t)b * (kBuckets + 1) + kBuckets] = n;
    // segments (a segment never crosses a sub-bucket).  Per sub-bucket, in
    // rounds of 32 keys: lane l holds key s0 + r + l; starts come from a
    // ballot, the carry is the open segment of the previous round.
    // Pass 0 counts the shared and long segments, pass 1 writes.
    for (int pass = 0; pass < 2; ++pass) {
        uint32_t n_m = 0, n_l = 0;
        for (int sb = warp; sb < kSub; sb += kWarps) {
            const uint32_t s0 = s_start[sb], c = s_start[sb + 1] - s0;
            for (uint32_t r = 0; r < c; r += 32) {
                const uint32_t i = s0 + r + lane;
                const bool valid = r + lane < c;
                const uint64_t key = valid ? a[i] : ~0ull;
                const uint32_t hk = (uint32_t)(key >> 32);
                const uint32_t prev = (valid && i > s0) ? (uint32_t)(a[i - 1] >> 32) : ~hk;
                const bool start = valid && prev != hk;
                const uint32_t smask = __ballot_sync(0xFFFFFFFFu, start);
                // each key's segment: first start at or below it (or the
                // round's carry), next start above it (or the sub-bucket end)
                const uint32_t below = smask & (0xFFFFFFFFu >> (31 - lane));
                uint32_t head = below ? s0 + r + (31 - __clz(below)) : 0u;
                uint32_t len = 0;
                if (valid) {
                    if (!below) {  // continues a segment of an earlier round (a hot row)
                        uint32_t h0 = i;
                        while (h0 > s0 && (uint32_t)(a[h0 - 1] >> 32) == hk) --h0;
                        head = h0;
                    }
                    const uint32_t above = smask & ~(0xFFFFFFFFu >> (31 - lane));
                    uint32_t end = above ? s0 + r + (__ffs(above) - 1) : 0u;
                    if (!above) {
                        end = s0 + min(c, r + 32);
                        while (end < s0 + c && (uint32_t)(a[end] >> 32) == hk) ++end;
                    }
                    len = end - head;
                }
                const bool is_head = valid && i == head;
                if (pass == 0) {
                    n_m += is_head && len > 1;
                    n_l += is_head && len > kChunk;
                    continue;
                }
                const uint32_t hpos = (uint32_t)(gpos + head);
                if (valid) {
                    const uint32_t v = (uint32_t)key;
                    const uint32_t slot = v & kSlotMask;
                    const uint32_t pos = (uint32_t)(gpos + i);
                    q.slot_info[(v >> kSlotBits) * q.R + slot] = make_uint2(pos | (len == 1 ? kSingleBit : 0u), hpos);
                }
                if (is_head) {
                    if (len > 1) {
                        // pair count of the segment: K + 1 for a source entry, 1 otherwise
                        uint32_t cnt = 0;
                        for (uint32_t k = head; k < head + len; ++k)
                            cnt += ((uint32_t)a[k] & kSlotMask) == 0 ? q.K + 1 : 1u;
                        const uint32_t key_row = unhrow(hk);
                        uint32_t flagged = len;
                        if (len > kChunk) {
                            const uint32_t l = *sh.lbase + atomicAdd(sh.lcnt, 1u);
                            q.ldesc[(size_t)b * q.lcap + l] = make_uint4(hpos, len, key_row, cnt);
                            flagged |= kLongBit;
                        }
                        const uint32_t m = *sh.mbase + atomicAdd(sh.mcnt, 1u);
                        q.mdesc[(size_t)b * q.mcap + m] = make_uint4(hpos, flagged, key_row, cnt);
                    }
                }
            }
        }
        if (pass == 0) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                n_m += __shfl_xor_sync(0xFFFFFFFFu, n_m, o);
                n_l += __shfl_xor_sync(0xFFFFFFFFu, n_l, o);
            }
            if (threadIdx.x == 0) {
                *sh.mcnt = 0;
                *sh.lcnt = 0;
            }
            __syncthreads();
            if (lane == 0 && n_m) atomicAdd(sh.mcnt, n_m);
            if (lane == 0 && n_l) atomicAdd(sh.lcnt, n_l);
            __syncthreads();
            if (threadIdx.x == 0) {
                *sh.mbase = *sh.mcnt ? atomicAdd(q.mcount + b, *sh.mcnt) : 0u;
                *sh.lbase = *sh.lcnt ? atomicAdd(q.lcount + b, *sh.lcnt) : 0u;
                *sh.mcnt = 0;
                *sh.lcnt = 0;
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kGroupThreads) k_group_cluster(GroupParams q, int log_parts) {
    extern __shared__ uint64_t gkeys[];                      // kGroupCap keys
    __shared__ uint32_t s_cnt[1 << kGroupMaxLog][kSub];      // this slice: keys per (part, sub-bucket)
    __shared__ uint32_t s_pre[1 << kGroupMaxLog][kSub];      // keys of (part, sub) in lower ranks' slices
    __shared__ uint32_t s_off[1 << kGroupMaxLog][kSub];      // where this slice's next key of (part, sub) goes
    __shared__ uint32_t s_start[kSub + 1];                   // my part's sub-bucket starts
    __shared__ uint32_t s_tot[1 << kGroupMaxLog];            // keys per part
    __shared__ uint32_t s_big[kSub];                         // sub-buckets too large for one thread
    __shared__ uint32_t s_nbig, s_mcnt, s_lcnt, s_mbase, s_lbase;
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t P = 1u << log_parts, me = cl.block_rank();
    const int b = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t base;
    uint32_t n;
    batch_range(q, b, &base, &n);
    for (uint32_t i = threadIdx.x; i < P * kSub; i += blockDim.x) (&s_cnt[0][0])[i] = 0;
    if (threadIdx.x == 0) s_nbig = 0;
    __syncthreads();
    const uint32_t per = (n + P - 1) / P;
    const uint32_t lo = min(n, me * per), hi = min(n, lo + per);
    const int sub_shift = 24 - log_parts;
    // pass 1: counts of this slice
    for (uint32_t r = lo; r < hi; r += kGroupThreads * kGroupPerThread) {
        uint64_t it[kGroupPerThread];
#pragma unroll
        for (int k = 0; k < kGroupPerThread; ++k) {
            const uint32_t i = r + k * kGroupThreads + threadIdx.x;
            it[k] = i < hi ? q.items[base + i] : 0ull;
        }
#pragma unroll
        for (int k = 0; k < kGroupPerThread; ++k) {
            const uint32_t i = r + k * kGroupThreads + threadIdx.x;
            if (i < hi) {
                const uint32_t hv = hrow((uint32_t)(it[k] >> 32));
                const uint32_t pt = log_parts ? hv >> (32 - log_parts) : 0u;
                atomicAdd(&s_cnt[pt][(hv >> sub_shift) & (kSub - 1)], 1u);
                if (q.depmap) {
                    const uint32_t db = hv >> (32 - kDepLog);
                    atomicOr(q.depmap + (size_t)b * kDepWords + (db >> 5), 1u << (db & 31u));
                }
            }
        }
    }
    cl.sync();
    // every (part, sub-bucket): total over the cluster, and the keys of lower
    // ranks (which go first); then per part the sub-bucket starts
    for (uint32_t e = threadIdx.x; e < P * kSub; e += blockDim.x) {
        uint32_t c[1 << kGroupMaxLog];
#pragma unroll
        for (uint32_t rk = 0; rk < (1u << kGroupMaxLog); ++rk)  // all loads in flight at once
            c[rk] = rk < P ? cl.map_shared_rank(&s_cnt[0][0], rk)[e] : 0u;
        uint32_t tot = 0, before = 0;
#pragma unroll
        for (uint32_t rk = 0; rk < (1u << kGroupMaxLog); ++rk) {
            if (rk < me) before += c[rk];
            tot += c[rk];
        }
        (&s_off[0][0])[e] = tot;  // totals for now
        (&s_pre[0][0])[e] = before;
    }
    __syncthreads();
    if (warp < (int)P) {
        // exclusive scan of part `warp`'s sub-bucket totals: lane l owns 8
        uint32_t v[kSub / 32], own = 0;
#pragma unroll
        for (int k = 0; k < kSub / 32; ++k) own += (v[k] = s_off[warp][lane * (kSub / 32) + k]);
        uint32_t incl = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += x;
        }
        uint32_t run = incl - own;
#pragma unroll
        for (int k = 0; k < kSub / 32; ++k) {
            const int sb = lane * (kSub / 32) + k;
            if (warp == (int)me) s_start[sb] = run;
            s_off[warp][sb] = run + s_pre[warp][sb];
            run += v[k];
        }
        if (lane == 31) {
            s_tot[warp] = run;
            if (warp == (int)me) s_start[kSub] = run;
        }
    }
    __syncthreads();
    uint32_t qbase = 0, pbase[1 << kGroupMaxLog];
    bool fits[1 << kGroupMaxLog];
    for (uint32_t p2 = 0, run = 0; p2 < P; ++p2) {
        pbase[p2] = run;
        if (p2 == me) qbase = run;
        fits[p2] = s_tot[p2] <= kGroupCap;
        run += s_tot[p2];
    }
    const uint32_t nq = s_tot[me];
    // pass 2: send every key to its place (a part too large for shared memory
    // - a very skewed draw - uses its own range of the scratch array)
    for (uint32_t r = lo; r < hi; r += kGroupThreads * kGroupPerThread) {
        uint64_t it[kGroupPerThread];
#pragma unroll
        for (int k = 0; k < kGroupPerThread; ++k) {
            const uint32_t i = r + k * kGroupThreads + threadIdx.x;
            it[k] = i < hi ? q.items[base + i] : 0ull;
        }
#pragma unroll
        for (int k = 0; k < kGroupPerThread; ++k) {
            const uint32_t i = r + k * kGroupThreads + threadIdx.x;
            if (i < hi) {
                const uint32_t hv = hrow((uint32_t)(it[k] >> 32));
                const uint32_t pt = log_parts ? hv >> (32 - log_parts) : 0u;
                const uint32_t at = atomicAdd(&s_off[pt][(hv >> sub_shift) & (kSub - 1)], 1u);
                uint64_t* dst = fits[pt] ? cl.map_shared_rank(gkeys, pt) : q.bucketed + base + pbase[pt];
                dst[at] = ((uint64_t)hv << 32) | (uint32_t)it[k];
            }
        }
    }
    cl.sync();
    const GroupShared sh{s_start, s_big, &s_nbig, &s_mcnt, &s_lcnt, &s_mbase, &s_lbase};
    if (fits[me]) group_tail(q, gkeys, nq, n, qbase, b, me, P, log_parts, sh);
    else group_tail(q, q.bucketed + base + qbase, nq, n, qbase, b, me, P, log_parts, sh);
}

// eta[b] = lr0 (schedule 0) or lr0 * max(1 - t0/T, floor) (schedule 1) for
// the batch starting at global sample t0 = t_chunk + b * batch, in FP32:
// 1 - t0/T as (T - t0) / T from the exact integer difference.
__global__ void k_batch_eta(int n_batches, uint64_t t_chunk, int64_t batch, float lr0, int schedule, float floor_frac,
                            uint64_t total, float* __restrict__ eta) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_batches) return;
    float f = 1.0f;
    if (schedule == 1) {
        const uint64_t t0 = t_chunk + (uint64_t)b * (uint64_t)batch;
        f = t0 >= total ? 0.0f : (float)(total - t0) / (float)total;
        if (f < floor_frac) f = floor_frac;
    }
    eta[b] = lr0 * f;
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

// Per-chunk outputs of the pre-pass, read by the data phase.  Two sets: the
// pre-pass of chunk c+1 (on its own low-priority stream) fills one while the
// data phase of chunk c reads the other.
struct ChunkSet {
    Buf rec, slot_info, depmap, mdesc, mcount, ldesc, lcount, eta, tchunk;
    // captured data phase of a full chunk of this set, and what it was
    // captured for: the parameters, the warps per block and the kernels (the
    // launcher of one row width and table type: tables of another type can
    // sit at the same addresses)
    cudaGraphExec_t graph = nullptr;
    DataParams graph_key{};
    int graph_wpb = -1;
    cudaError_t (*graph_fn)(const DataParams&, int, cudaStream_t) = nullptr;
    cudaEvent_t prep_done = nullptr;  // pre-pass of the set's current chunk finished
    cudaEvent_t data_done = nullptr;  // data phase of the set's previous chunk finished
    bool data_pending = false;
};

struct TrainWorkspace {
    Buf items0, items1, gcnt, boff, counters, slab, gbar;
    ChunkSet set[2];
    cudaStream_t prep = nullptr;    // pre-pass stream
    cudaStream_t cap = nullptr;     // stream the data-phase graphs are captured on
    bool graph_failed = false;      // a capture failed: direct launches from then on
    cudaEvent_t start = nullptr;    // caller-stream work before the call
    cudaEvent_t prep_end = nullptr; // last pre-pass of the call
    std::vector<cudaEvent_t> events;  // timing events
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
    cudaError_t init(int device) {
        if (prep) return cudaSuccess;
        int lo = 0, hi = 0;
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&prep, cudaStreamNonBlocking, lo);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        for (auto& cs : set) {
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&cs.prep_done, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&cs.data_done, cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&prep_end, cudaEventDisableTiming);
        (void)device;
        return e;
    }
    ~TrainWorkspace() {
        if (prep) {
            cudaStreamSynchronize(prep);
            cudaStreamDestroy(prep);
        }
        if (cap) cudaStreamDestroy(cap);
        for (auto& cs : set) {
            if (cs.prep_done) cudaEventDestroy(cs.prep_done);
            if (cs.data_done) cudaEventDestroy(cs.data_done);
            if (cs.graph) cudaGraphExecDestroy(cs.graph);
        }
        if (start) cudaEventDestroy(start);
        if (prep_end) cudaEventDestroy(prep_end);
        for (auto e : events) cudaEventDestroy(e);
    }
};

TrainWorkspace* workspace_create() { return new TrainWorkspace(); }
void workspace_destroy(TrainWorkspace* ws) { delete ws; }

static uint32_t bits_for(uint64_t v) {  // bits to hold values 0..v-1
    uint32_t b = 1;
    while ((1ull << b) < v) ++b;
    return b;
}

// Runs f once per device (function attributes are per device); thread-safe.
template <typename F>
static void once_per_device(std::atomic<uint64_t>& done, F f) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    const uint64_t bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    f();
    done.fetch_or(bit, std::memory_order_acq_rel);
}

template <int D, int DT>
static int gather_warps(const DataParams& p, int requested, int cap, size_t* smem_out, int dflt = 8) {
    using G = Geom<D, DT>;
    // staging: (K+1) context rows x 32 lanes x E floats per warp
    const size_t per_warp = (size_t)(p.K + 1) * 32 * G::E * sizeof(float);
    int wpb = requested > 0 ? requested : dflt;
    wpb = std::min<int>(wpb, cap);
    wpb = std::max<int>(1, std::min<int>(wpb, (int)(kMaxSmem / per_warp)));
    *smem_out = (size_t)wpb * per_warp;
    return wpb;
}

template <typename... Args, typename... Vals>
static cudaError_t launch_pdl(void (*kern)(Args...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                              bool pdl, Vals... vals) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, vals...);
}

template <int D, int DT>
static cudaError_t launch_data_batched(const DataParams& p, int warps_per_block, cudaStream_t s) {
    using G = Geom<D, DT>;
    size_t smem = 0;
    // 4 warps per block: at ~70 registers a 4096-sample batch is one wave
    const int wpb = gather_warps<D, DT>(p, warps_per_block, kGatherWarps, &smem, kGatherWarps);
    static std::atomic<uint64_t> attr_set{0};
    once_per_device(attr_set, [] {
        cudaFuncSetAttribute(k_gather<D, DT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
        cudaFuncSetAttribute(k_gather<D, DT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    });
    const int64_t per_block = (int64_t)wpb * G::GPW;
    const int aw = p.apply_warps == kApplyWarpsAlone ? kApplyWarpsAlone : kApplyWarpsShared;
    const int64_t apply_per_block = (int64_t)aw * G::GPW;
    // long shared segments (more than kChunk entries, ~34 per batch on R-MAT 20)
    // each get a CTA of their own
    const int g_long = 64;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < p.n_batches && e == cudaSuccess; ++b) {
        const int64_t nb = std::min<int64_t>(p.batch, p.chunk_samples - (int64_t)b * p.batch);
        const unsigned g1 = (unsigned)((nb + per_block - 1) / per_block);
        // the chunk's first gather follows the pre-pass with a full dependency;
        // later launches overlap their start with the previous kernel's tail
        if (b == 0) e = launch_pdl(k_gather<D, DT, false>, g1, wpb * 32, smem, s, false, p, b);
        else e = launch_pdl(k_gather<D, DT, true>, g1, wpb * 32, smem, s, true, p, b);
        if (e != cudaSuccess) break;
        // a shared segment has two or more of the batch's nb * (K+2) entries
        const int64_t max_m = nb * (p.K + 2) / 2 + 1;
        // short shared segments run about 10% of the batch's entries (R-MAT
        // 20: ~2.9K of 28.7K); 2 blocks per SM leave room for the next kernel
        const unsigned g2 = (unsigned)std::min<int64_t>((max_m + apply_per_block - 1) / apply_per_block, 152 * 2);
        if (aw == kApplyWarpsAlone)
            e = launch_pdl(k_apply<D, DT, kApplyWarpsAlone>, (unsigned)g_long + g2, kApplyWarpsAlone * 32, 0, s, true, p,
                           b, g_long);
        else
            e = launch_pdl(k_apply<D, DT, kApplyWarpsShared>, (unsigned)g_long + g2, kApplyWarpsShared * 32, 0, s, true,
                           p, b, g_long);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int D, int DT>
static cudaError_t launch_data_persistent(const DataParams& p, int warps_per_block, cudaStream_t s) {
    using G = Geom<D, DT>;
    int dev = 0, sms = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    int W = warps_per_block > 0 ? std::min(warps_per_block, kPersistMaxWarps) : kPersistDefaultWarps;
    // two row slots per warp when a warp has two or more units of a batch
    auto slots_for = [&](int w) {
        const int64_t units = (p.batch + G::GPW - 1) / G::GPW;
        return units > (int64_t)sms * w ? 2 : 1;
    };
    size_t smem = persist_smem_bytes(D, DT, p.K, W, slots_for(W), G::GPW);
    while (W > 1 && smem > (size_t)optin) {
        --W;
        smem = persist_smem_bytes(D, DT, p.K, W, slots_for(W), G::GPW);
    }
    if (smem > (size_t)optin) return cudaErrorInvalidConfiguration;
    if ((e = cudaFuncSetAttribute(k_persistent<D, DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent<D, DT>, W * 32, smem)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    DataParams pc = p;
    pc.slots = slots_for(W);
    if ((e = cudaMemsetAsync(p.gbar, 0, 2 * sizeof(uint32_t), s)) != cudaSuccess) return e;
    void* args[] = {&pc};
    return cudaLaunchCooperativeKernel((const void*)k_persistent<D, DT>, dim3((unsigned)sms), dim3((unsigned)(W * 32)),
                                       args, smem, s);
}

using LaunchFn = cudaError_t (*)(const DataParams&, int, cudaStream_t);

static LaunchFn pick_launcher(int dim, int dtype, bool persistent) {
#define LINE_PICK(DD)                                                                                   \
    if (dim == DD) {                                                                                    \
        if (persistent)                                                                                 \
            return dtype == LINE_DTYPE_F32 ? launch_data_persistent<DD, LINE_DTYPE_F32>                 \
                                           : launch_data_persistent<DD, LINE_DTYPE_BF16>;               \
        return dtype == LINE_DTYPE_F32 ? launch_data_batched<DD, LINE_DTYPE_F32>                        \
                                       : launch_data_batched<DD, LINE_DTYPE_BF16>;                      \
    }
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
        *err = "too many nodes for 32-bit row ids";
        return cudaErrorInvalidValue;
    }
    // batches per chunk: about 2^18 samples (2^20 for walk pairs in the
    // Hogwild schedule, whose faster update launch would otherwise wait for
    // the next chunk's walks: a walk's steps are sequential, so a chunk's
    // walks take about the same time whatever their number), limited by
    // 31-bit positions and by the chunk-sample field of item values
    const bool long_chunks = a.mode == LINE_MODE_HOGWILD && a.walk_len > 0;
    int64_t nb = a.chunk_batches > 0 ? a.chunk_batches
                                     : std::max<int64_t>(1, (int64_t(1) << (long_chunks ? 20 : 18)) / a.batch);
    while (nb > 1 && ((uint64_t)nb * (uint64_t)a.batch * (uint64_t)R >= (1ull << 31) ||
                      (uint64_t)nb * (uint64_t)a.batch > (1ull << (32 - kSlotBits))))
        nb >>= 1;
    const uint64_t total_batches = (n_samples + a.batch - 1) / a.batch;
    nb = (int64_t)std::min<uint64_t>((uint64_t)nb, total_batches);
    const int64_t max_chunk = nb * a.batch;
    const int64_t max_items = max_chunk * R;
    const uint32_t parts = (uint32_t)((a.batch * R + kPartItems - 1) / kPartItems);
    // batches of up to 8 parts of ~3.5K items are grouped by one cluster in
    // distributed shared memory; larger ones are bucketed through global
    // memory first
    int log_parts = 0;
    while (a.batch * R > ((int64_t)3584 << log_parts)) ++log_parts;
    const bool direct = log_parts <= kGroupMaxLog;
    // the persistent schedule needs all its CTAs resident at once, which a
    // second cooperative launch on the other order's stream could prevent:
    // concurrent orders run the batched schedule
    const bool persistent = a.mode == LINE_MODE_PERSISTENT && !a.concurrent;
    const bool hogwild = a.mode == LINE_MODE_HOGWILD;  // records only: no grouping, slab or apply
    // shared segments (two or more entries) and long ones (more than kChunk)
    // per batch, at most
    const uint32_t mcap = (uint32_t)(a.batch * R / 2 + 1);
    const uint32_t lcap = (uint32_t)(a.batch * R / (kChunk + 1) + 1);

    cudaError_t e;
    auto ensure = [&](Buf& b, size_t bytes) -> bool {
        if ((e = b.ensure(bytes)) != cudaSuccess) {
            *err = "device allocation failed (training scratch)";
            return false;
        }
        return true;
    };
    int device = 0;
    if ((e = cudaGetDevice(&device)) != cudaSuccess) return e;
    if ((e = ws->init(device)) != cudaSuccess) return e;
    // every scratch buffer and its size for this call
    auto each = [&](auto&& f) -> bool {
        if (hogwild) {
            for (auto& cs : ws->set)
                if (!f(cs.rec, sizeof(int32_t) * max_items) || !f(cs.tchunk, 256)) return false;
            return true;
        }
        if (!f(ws->items0, sizeof(uint64_t) * max_items) || !f(ws->items1, sizeof(uint64_t) * max_items) ||
            !f(ws->gcnt, sizeof(uint32_t) * (size_t)nb * parts * kBuckets) ||
            !f(ws->boff, sizeof(uint32_t) * (size_t)nb * (kBuckets + 1)) || !f(ws->counters, 256) ||
            !f(ws->slab, sizeof(float) * (size_t)std::min<int64_t>(max_items, a.batch * R) * a.dim))
            return false;
        for (auto& cs : ws->set) {
            if (!f(cs.rec, sizeof(int32_t) * max_items) || !f(cs.eta, sizeof(float) * (nb + 1)) ||
                !f(cs.slot_info, sizeof(uint2) * max_items) || !f(cs.mdesc, sizeof(uint4) * (size_t)nb * mcap) ||
                !f(cs.mcount, sizeof(uint32_t) * (nb + 1)) || !f(cs.ldesc, sizeof(uint4) * (size_t)nb * lcap) ||
                !f(cs.lcount, sizeof(uint32_t) * (nb + 1)) || !f(cs.tchunk, 256))
                return false;
            if (persistent && !f(cs.depmap, sizeof(uint32_t) * (size_t)nb * kDepWords)) return false;
        }
        return true;
    };
    // Buffers still used by an earlier call's data phase are reallocated
    // only after that phase is done; when nothing grows, consecutive calls on
    // the stream pipeline (the chunk sets' events order the reuse).
    bool grow = false;
    each([&](Buf& b, size_t bytes) {
        grow = grow || b.cap < bytes;
        return true;
    });
    if (grow) {
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        if (ws->prep && (e = cudaStreamSynchronize(ws->prep)) != cudaSuccess) return e;
        for (auto& cs : ws->set) cs.data_pending = false;
        if (!each(ensure)) return e;
    }
    if (persistent && !ensure(ws->gbar, 256)) return e;
    LaunchFn data = pick_launcher(a.dim, a.dtype, persistent);
    if (!data) {
        *err = "unsupported dim";
        return cudaErrorInvalidValue;
    }
    const size_t sort_smem = (size_t)kSortBucketsPerCta * 2 * kWarpSortCap * sizeof(uint64_t);
    const size_t group_smem = (size_t)kGroupCap * sizeof(uint64_t);
    if ((e = cudaFuncSetAttribute(k_bucket_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_group_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)group_smem)) !=
            cudaSuccess)
        return e;
    cudaStream_t ps = ws->prep;
    // the pre-pass reads the graph and alias tables made on the caller's stream
    if ((e = cudaEventRecord(ws->start, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(ps, ws->start, 0)) != cudaSuccess) return e;

    PrepassParams pp{};
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
    pp.walk = a.walk_len > 0;
    pp.items = hogwild ? nullptr : (uint64_t*)ws->items0.p;

    WalkParams wp{};
    if (a.walk_len > 0) {
        wp.src = a.src;
        wp.dst = a.dst;
        wp.edge_tab = a.edge_tab;
        wp.n_arcs = a.n_arcs;
        wp.row_ptr = a.row_ptr;
        wp.cw = a.cw;
        wp.seed = a.seed;
        wp.L = a.walk_len;
        wp.W = a.window;
        wp.P = (uint64_t)a.walk_len * a.window - (uint64_t)a.window * (a.window - 1) / 2;
        wp.reuse = (uint32_t)a.walk_reuse;
        wp.R = (uint64_t)R;
        wp.items = hogwild ? nullptr : (uint64_t*)ws->items0.p;
        wp.ctx_off = a.order == 2 ? (uint32_t)a.n_nodes : 0u;
        wp.slot_bits = kSlotBits;
    }

    GroupParams gq{};
    gq.batch = a.batch;
    gq.R = (uint32_t)R;
    gq.K = (uint32_t)a.K;
    gq.parts = parts;
    gq.row_bits = row_bits;
    gq.items = (const uint64_t*)ws->items0.p;
    gq.bucketed = (uint64_t*)ws->items1.p;
    gq.tmp = (uint64_t*)ws->items0.p;  // the draws are consumed by the bucketing before the sort
    gq.gcnt = (uint32_t*)ws->gcnt.p;
    gq.boff = (uint32_t*)ws->boff.p;
    gq.mcap = mcap;
    gq.lcap = lcap;

    uint32_t* abort_word = (uint32_t*)ws->counters.p + 16;

    DataParams dp{};
    dp.U = a.U;
    dp.C = a.order == 2 ? a.C : a.U;
    dp.order = a.order;
    dp.K = a.K;
    dp.n_nodes = a.n_nodes;
    dp.row_bits = row_bits;
    dp.mcap = mcap;
    dp.lcap = lcap;
    dp.slab = (float*)ws->slab.p;
    dp.batch = a.batch;
    dp.seed = a.seed;
    dp.lambda = (float)a.lambda;
    dp.alpha_neg = (float)a.alpha_neg;
    dp.status = status;
    dp.gbar = (uint32_t*)ws->gbar.p;
    dp.spin_limit = a.spin_limit;
    dp.abort_word = abort_word;
    dp.apply_warps = a.concurrent ? kApplyWarpsShared : kApplyWarpsAlone;

    struct ChunkRec {
        size_t ev;  // events ev, ev+1 (pre-pass stream), ev+2, ev+3 (data stream)
    };
    std::vector<ChunkRec> chunk_log;
    size_t n_ev = 0;
    cudaEvent_t ev = nullptr;
    int c = 0;
    for (uint64_t t = a.t_begin; t < a.t_end; t += (uint64_t)max_chunk, ++c) {
        ChunkSet& cset = ws->set[c & 1];
        const int64_t cs = (int64_t)std::min<uint64_t>((uint64_t)max_chunk, a.t_end - t);
        const int cb = (int)((cs + a.batch - 1) / a.batch);
        const int64_t n_items = cs * R;
        int launches = 0;
        // ---- pre-pass of chunk c on the pre-pass stream, into set c % 2,
        // once the data phase of chunk c-2 (the set's last reader) is done
        if (cset.data_pending && (e = cudaStreamWaitEvent(ps, cset.data_done, 0)) != cudaSuccess) return e;
        if (a.timing) {
            if ((e = ws->event(n_ev, &ev)) != cudaSuccess) return e;
            cudaEventRecord(ev, ps);
        }
        pp.t_chunk = t;
        pp.chunk_samples = cs;
        pp.rec = (int32_t*)cset.rec.p;
        pp.t_out = (uint64_t*)cset.tchunk.p;
        {
            const int64_t work = cs * (a.K + 1);
            const unsigned g = (unsigned)std::min<int64_t>((work + 255) / 256, 152 * 64);
            k_chunk_draws<<<g, 256, 0, ps>>>(pp);
            if (a.walk_len > 0) {
                wp.t0 = t;
                wp.count = cs;
                wp.rec = (int32_t*)cset.rec.p;
                if ((e = walk_pairs(wp, ps)) != cudaSuccess) return e;
                ++launches;
            }
            if (!hogwild)
                k_batch_eta<<<(unsigned)((cb + 127) / 128), 128, 0, ps>>>(cb, t, a.batch, (float)a.lr0, a.lr_schedule,
                                                                          (float)a.lr_floor, a.lr_total,
                                                                          (float*)cset.eta.p);
        }
        if (!hogwild) {
            gq.n_batches = cb;
            gq.chunk_samples = cs;
            gq.slot_info = (uint2*)cset.slot_info.p;
            gq.mdesc = (uint4*)cset.mdesc.p;
            gq.mcount = (uint32_t*)cset.mcount.p;
            gq.ldesc = (uint4*)cset.ldesc.p;
            gq.lcount = (uint32_t*)cset.lcount.p;
            gq.depmap = persistent ? (uint32_t*)cset.depmap.p : nullptr;
            if ((e = cudaMemsetAsync(cset.mcount.p, 0, sizeof(uint32_t) * (cb + 1), ps)) != cudaSuccess) return e;
            if ((e = cudaMemsetAsync(cset.lcount.p, 0, sizeof(uint32_t) * (cb + 1), ps)) != cudaSuccess) return e;
            if (persistent &&
                (e = cudaMemsetAsync(cset.depmap.p, 0, sizeof(uint32_t) * (size_t)cb * kDepWords, ps)) != cudaSuccess)
                return e;
            if (direct) {
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(1u << log_parts, cb);
                cfg.blockDim = dim3(kGroupThreads);
                cfg.dynamicSmemBytes = group_smem;
                cfg.stream = ps;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = 1u << log_parts;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                if ((e = cudaLaunchKernelEx(&cfg, k_group_cluster, gq, log_parts)) != cudaSuccess) return e;
                launches += 3;
            } else {
                k_bucket_count<<<dim3(parts, cb), kBucketThreads, 0, ps>>>(gq);
                k_bucket_scatter<<<dim3(parts, cb), kBucketThreads, 0, ps>>>(gq);
                k_bucket_sort<<<dim3(kBuckets / kSortBucketsPerCta, cb), kSortThreads, sort_smem, ps>>>(gq);
                launches += 5;
            }
        } else {
            launches += 1;  // the draws alone
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (a.timing) {
            if ((e = ws->event(n_ev + 1, &ev)) != cudaSuccess) return e;
            cudaEventRecord(ev, ps);
        }
        if ((e = cudaEventRecord(cset.prep_done, ps)) != cudaSuccess) return e;
        // ---- data phase of chunk c on the caller's stream
        if ((e = cudaStreamWaitEvent(s, cset.prep_done, 0)) != cudaSuccess) return e;
        if (a.timing) {
            if ((e = ws->event(n_ev + 2, &ev)) != cudaSuccess) return e;
            cudaEventRecord(ev, s);
        }
        if (hogwild) {
            HogwildParams hp{};
            hp.U = a.U;
            hp.C = a.C;
            hp.order = a.order;
            hp.K = a.K;
            hp.n_nodes = a.n_nodes;
            hp.rec = (const int32_t*)cset.rec.p;
            hp.chunk_samples = cs;
            hp.t_chunk = t;
            hp.batch = a.batch;
            hp.lr0 = (float)a.lr0;
            hp.lr_floor = (float)a.lr_floor;
            hp.lr_schedule = a.lr_schedule;
            hp.lr_total = a.lr_total;
            hp.lambda = (float)a.lambda;
            hp.alpha_neg = (float)a.alpha_neg;
            hp.seed = a.seed;
            hp.status = status;
            if ((e = hogwild_chunk(hp, a.dim, a.dtype, a.hogwild_workers, s)) != cudaSuccess) return e;
        } else {
            dp.rec = (const int32_t*)cset.rec.p;
            dp.slot_info = (const uint2*)cset.slot_info.p;
            dp.mdesc = (const uint4*)cset.mdesc.p;
            dp.mcount = (const uint32_t*)cset.mcount.p;
            dp.ldesc = (const uint4*)cset.ldesc.p;
            dp.lcount = (const uint32_t*)cset.lcount.p;
            dp.eta = (const float*)cset.eta.p;
            dp.depmap = (const uint32_t*)cset.depmap.p;
            dp.t_chunk = t;
            dp.chunk_samples = cs;
            dp.n_batches = cb;
            if (persistent && (e = cudaMemsetAsync(abort_word, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
            if (!persistent && a.graph && !ws->graph_failed && cs == max_chunk && c > 0) {
                // a full chunk: replay this set's captured data phase (the chunk's
                // first sample index comes from the set's device copy)
                dp.t_chunk_dev = (const uint64_t*)cset.tchunk.p;
                DataParams key = dp;
                key.t_chunk = 0;
                if (!cset.graph || cset.graph_wpb != a.warps_per_block || cset.graph_fn != data ||
                    memcmp(&key, &cset.graph_key, sizeof key) != 0) {
                    if (cset.graph) cudaGraphExecDestroy(cset.graph);
                    cset.graph = nullptr;
                    cudaGraph_t g = nullptr;
                    cudaError_t ce = cudaStreamBeginCapture(ws->cap, cudaStreamCaptureModeThreadLocal);
                    if (ce == cudaSuccess) {
                        const cudaError_t le = data(dp, a.warps_per_block, ws->cap);
                        ce = cudaStreamEndCapture(ws->cap, &g);
                        if (ce == cudaSuccess) ce = le;
                    }
                    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&cset.graph, g, 0);
                    if (g) cudaGraphDestroy(g);
                    if (ce != cudaSuccess) {
                        cudaGetLastError();
                        cset.graph = nullptr;
                        ws->graph_failed = true;
                    } else {
                        cset.graph_key = key;
                        cset.graph_wpb = a.warps_per_block;
                        cset.graph_fn = data;
                    }
                }
                if (cset.graph) {
                    if ((e = cudaGraphLaunch(cset.graph, s)) != cudaSuccess) return e;
                } else {
                    dp.t_chunk_dev = nullptr;
                    if ((e = data(dp, a.warps_per_block, s)) != cudaSuccess) return e;
                }
            } else {
                dp.t_chunk_dev = nullptr;
                if ((e = data(dp, a.warps_per_block, s)) != cudaSuccess) return e;
            }
        }
        if (a.timing) {
            if ((e = ws->event(n_ev + 3, &ev)) != cudaSuccess) return e;
            cudaEventRecord(ev, s);
            chunk_log.push_back({n_ev});
            n_ev += 4;
        }
        if ((e = cudaEventRecord(cset.data_done, s)) != cudaSuccess) return e;
        cset.data_pending = true;
        // launches counted whether or not they are timed (a graph replay
        // counts the kernels it holds)
        times->prepass_launches += launches;
        times->update_launches += (persistent || hogwild) ? 1 : 2 * (int64_t)cb;
        times->update_samples += (uint64_t)cs;
    }
    // the pre-pass stream's work is all ordered before the last data phase
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (a.timing && n_ev) {
        if ((e = cudaEventSynchronize(ws->events[n_ev - 1])) != cudaSuccess) return e;
        for (const ChunkRec& r : chunk_log) {
            float ms1 = 0, ms2 = 0;
            cudaEventElapsedTime(&ms1, ws->events[r.ev], ws->events[r.ev + 1]);
            cudaEventElapsedTime(&ms2, ws->events[r.ev + 2], ws->events[r.ev + 3]);
            times->prepass_ms += ms1;
            times->update_ms += ms2;
        }
    }
    return cudaSuccess;
}

}  // namespace line
