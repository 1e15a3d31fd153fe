// Internal declarations of the LINE library (device helpers, kernel launchers,
// the context).  Not part of the public ABI (include/line.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "line.h"

namespace line {

// ---------------------------------------------------------------------------
// Status word bits written by kernels (never __trap: a kernel that hits one of
// these records it and returns; the host turns the word into a status).
// ---------------------------------------------------------------------------
enum : uint32_t {
    DEV_ERR_INDEX = 1u << 0,    // an index read from memory was out of range
    DEV_ERR_TIMEOUT = 1u << 1,  // a bounded wait ran out
    DEV_ERR_GRAPH = 1u << 2,    // graph validation failed
    DEV_ERR_ALIAS = 1u << 3,    // alias construction invariant failed
    DEV_ERR_VALUE = 1u << 4,    // a computed value was not finite
};

constexpr uint64_t kQ = 1ull << 32;
constexpr uint32_t kThrFull = 0xFFFFFFFFu;
constexpr int kMaxK = 32;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32
// S-box with multipliers 0xD2511F53 / 0xCD9E8D57, key bumped by the Weyl
// constants 0x9E3779B9 / 0xBB67AE85 between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw_words(uint64_t seed, uint32_t domain, uint64_t t, uint32_t call) {
    return philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), call, domain),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Alias table entry: x = threshold, y = alias.  i = mulhi64(w1:w0, n);
// keep i when w2 < thr[i], else take alias[i].
__device__ __forceinline__ uint32_t alias_pick(const uint2* __restrict__ tab, uint64_t n, uint4 w) {
    const uint64_t r = ((uint64_t)w.y << 32) | (uint64_t)w.x;
    const uint64_t i = __umul64hi(r, n);
    const uint2 e = __ldg(tab + i);
    return w.z < e.x ? (uint32_t)i : e.y;
}

// Cache-global (L2, not L1) vector loads/stores: rows written by other SMs
// during a persistent launch must not be served from a stale L1 line.
__device__ __forceinline__ float4 ld_cg(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ uint4 ld_cg(const uint4* p) { return __ldcg(p); }
__device__ __forceinline__ void st_cg(float4* p, float4 v) { __stcg(p, v); }
__device__ __forceinline__ void st_cg(uint4* p, uint4 v) { __stcg(p, v); }

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t* p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void red_release_add(uint32_t* p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait until *flag >= target (unsigned compare).  Returns false when
// the limit ran out or another warp already reported a failure (abort word
// non-zero); the caller then records the failure and returns.
__device__ __forceinline__ bool wait_geq(const uint32_t* flag, uint32_t target, int64_t limit,
                                         const uint32_t* abort_word) {
    int64_t it = 0;
    uint32_t ns = 32;
    while (ld_acquire(flag) < target) {
        if (++it > limit || *(volatile const uint32_t*)abort_word) return false;
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
    }
    return true;
}

// Stochastic rounding FP32 -> BF16: add 16 random bits below the BF16
// mantissa, then truncate.  Inf and NaN pass through unchanged.
__device__ __forceinline__ uint16_t bf16_sr(float x, uint32_t r16) {
    uint32_t b = __float_as_uint(x);
    if ((b & 0x7F800000u) != 0x7F800000u) b += r16 & 0xFFFFu;
    return (uint16_t)(b >> 16);
}

// The same rounding of two values in one instruction: cvt.rs (stochastic
// rounding with explicit random bits) puts `hi` in the upper half of the
// result, rounded with bits [16, 32) of r, and `lo` in the lower half with
// bits [0, 16) - that is, bf16_sr(lo, r) | bf16_sr(hi, r >> 16) << 16, bit for
// bit on every input except the payload of a NaN (a NaN stays a NaN).
__device__ __forceinline__ uint32_t bf16x2_sr(float lo, float hi, uint32_t r) {
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    return d;
}

// ---------------------------------------------------------------------------
// Launchers (defined in the .cu files).  All enqueue on `s`.
// ---------------------------------------------------------------------------
struct DeviceScratch {
    void* p = nullptr;
    size_t bytes = 0;
};

// alias.cu
// Block of the fixed-order FP64 sum: blocks of kSumBlock values are each
// reduced by halving strides, then the block sums likewise, recursively.
constexpr int kSumBlock = 1024;
cudaError_t fixed_sum_f64(const double* x, int64_t n, double* tmp, double* out, cudaStream_t s);
size_t fixed_sum_tmp_bytes(int64_t n);
cudaError_t validate_graph(int64_t n_nodes, int64_t n_arcs, const int32_t* src, const int32_t* dst,
                           const float* w, uint32_t* status, cudaStream_t s);
cudaError_t edge_weights(int64_t n_arcs, const float* w, double* x, cudaStream_t s);
// x[v] = d(v)^0.75; deg (nullable): d(v) rounded to FP32.  row_ptr: the
// first arc of each node (row_offsets).  flag: one word of device scratch.
cudaError_t neg_weights(int64_t n_nodes, int64_t n_arcs, const int64_t* row_ptr, const float* w, double* x, float* deg,
                        uint32_t* flag, cudaStream_t s);
size_t alias_build_tmp_bytes(int64_t n);
// Builds tab[n] = {thr, alias} from weights x[n] (FP64).  tmp: alias_build_tmp_bytes(n).
cudaError_t alias_build(const double* x, int64_t n, uint2* tab, void* tmp, uint32_t* status, cudaStream_t s);

// sample.cu
cudaError_t sample_records(const int32_t* src, const int32_t* dst, const uint2* edge_tab, int64_t n_arcs,
                           const uint2* neg_tab, int64_t n_nodes, uint64_t seed, uint32_t domain,
                           uint64_t t0, int64_t count, int K, int32_t* out, cudaStream_t s);
cudaError_t export_alias(const uint2* tab, int64_t n, uint32_t* thr, uint32_t* alias, cudaStream_t s);
cudaError_t init_table(void* U, int dtype, int64_t n, int dim, uint64_t seed, cudaStream_t s);
cudaError_t convert_rows(const void* src, int src_dtype, void* dst, int dst_dtype, const int32_t* rows,
                         int64_t n_rows, int dim, int64_t n_nodes, uint32_t* status, cudaStream_t s);
cudaError_t debug_wait(uint32_t* flag, int64_t limit, uint32_t* status, cudaStream_t s);

// walk.cu: the walk sampler (Algorithms 2-3).  Limits: 1 <= W <= L <= kMaxWalkLen,
// 1 <= reuse <= kMaxWalkReuse.
constexpr int kMaxWalkLen = 1024;
constexpr int kMaxWalkReuse = 1024;
struct WalkParams {
    const int32_t* src;
    const int32_t* dst;
    const uint2* edge_tab;
    int64_t n_arcs;
    const int64_t* row_ptr;  // [n_nodes + 1]
    const double* cw;        // [n_arcs] running weight sums per node
    uint64_t seed;
    uint64_t t0;             // global index of the first sample
    int64_t count;
    int L, W;
    uint64_t P;              // pairs per walk: L W - W (W - 1) / 2
    uint32_t reuse;          // passes over each walk's pairs (>= 1)
    uint64_t R;              // record stride (K + 2)
    int32_t* rec;            // rec[s R], rec[s R + 1] = the pair of sample t0 + s
    uint64_t* items;         // nullable: grouping items of slots 0 and 1
    uint32_t ctx_off;        // row offset of the context table in the items
    uint32_t slot_bits;      // item value = (s << slot_bits) | slot
};
size_t walk_smem_bytes(int L);
// row_ptr[n+1]: first arc of each node, from the sorted src.
cudaError_t row_offsets(int64_t n_nodes, int64_t n_arcs, const int32_t* src, int64_t* row_ptr, cudaStream_t s);
// cw[m]: running FP64 sums of each node's arc weights (w nullable: weight 1).
cudaError_t walk_cumw(int64_t n_nodes, const int64_t* row_ptr, const float* w, double* cw, cudaStream_t s);
cudaError_t walk_pairs(const WalkParams& p, cudaStream_t s);

// eval.cu
cudaError_t eval_loss_terms(const void* U, const void* Ctx, int dtype, int dim, int K, const int32_t* src,
                            const int32_t* dst, const uint2* edge_tab, int64_t n_arcs, const uint2* neg_tab,
                            int64_t n_nodes, uint64_t seed, int64_t m, double* terms, cudaStream_t s);

// auc.cu: link-prediction scores and AUC
struct ScoreTables {
    int n;  // number of tables (orders) concatenated, 1 or 2
    const void* U[2];
    int dim[2];
    int dtype[2];
};
size_t auc_tmp_bytes(int64_t n_pos, int64_t n_neg);
// src/dst: n_pos positive pairs then n_neg negative pairs (device).  scores:
// [n_pos + n_neg] FP32 out.  tmp: auc_tmp_bytes(n_pos, n_neg) bytes, 256-byte
// aligned; on return its first two u64 are {#(neg < pos), #(neg == pos)}.
cudaError_t eval_auc(const ScoreTables& t, int score, const int32_t* src, const int32_t* dst, int64_t n_pos, int64_t n_neg,
                     int64_t n_nodes, float* scores, void* tmp, uint32_t* status, cudaStream_t s);

// noalloc.cu: the loss evaluation with its scratch in a fixed device array
cudaError_t noalloc_scratch_address(int device, double** out);
cudaError_t eval_loss_noalloc(int device, const void* U, const void* Ctx, int dtype, int dim, int K,
                              const int32_t* src, const int32_t* dst, const uint2* edge_tab, int64_t n_arcs,
                              const uint2* neg_tab, int64_t n_nodes, uint64_t seed, int64_t m, double* out_dev,
                              cudaStream_t s);

// hogwild.cu: one chunk of the Hogwild schedule (per-pair immediate updates
// by concurrent lane-group workers) over the chunk's records.
struct HogwildParams {
    void* U;
    void* C;
    int order, K;
    int64_t n_nodes;
    const int32_t* rec;  // [chunk_samples][K+2]
    int64_t chunk_samples;
    uint64_t t_chunk;    // global index of the chunk's first sample (a batch start)
    int64_t batch;       // learning-rate steps
    float lr0, lr_floor;
    int lr_schedule;
    uint64_t lr_total;
    float lambda, alpha_neg;
    uint64_t seed;
    int64_t workers;     // set by the launcher
    uint32_t* status;
};
// max_workers <= 0: one resident wave of workers.
cudaError_t hogwild_chunk(const HogwildParams& p, int dim, int dtype, int64_t max_workers, cudaStream_t s);

// train.cu
struct TrainArgs {
    int order, dim, K, dtype;
    int64_t n_nodes, n_arcs;
    const int32_t* src;
    const int32_t* dst;
    const uint2* edge_tab;
    const uint2* neg_tab;
    void* U;
    void* C;
    uint64_t seed;
    uint64_t t_begin, t_end;  // global sample range of the call
    int64_t batch;
    double lr0, lr_floor;
    int lr_schedule;
    uint64_t lr_total;
    double lambda, alpha_neg;
    int mode;
    int64_t spin_limit;
    int chunk_batches;
    int warps_per_block;
    int timing;
    int graph;
    // walk sampler (walk_len > 0): positive pairs from random walks
    const int64_t* row_ptr;
    const double* cw;
    int walk_len, window, walk_reuse;
    int64_t hogwild_workers;  // LINE_MODE_HOGWILD: concurrent workers (0: one resident wave)
    bool concurrent;          // another order trains at the same time (line_train_orders)
};

struct TrainTimes {
    int64_t update_launches = 0;
    double update_ms = 0;
    uint64_t update_samples = 0;
    int64_t prepass_launches = 0;
    double prepass_ms = 0;
};

struct TrainWorkspace;  // scratch owned by the context (train.cu)
TrainWorkspace* workspace_create();
void workspace_destroy(TrainWorkspace*);
// Returns cudaSuccess or the first CUDA error; device-side failures are
// reported through *status (read by the caller after synchronising).
cudaError_t train_run(const TrainArgs& a, TrainWorkspace* ws, uint32_t* status, TrainTimes* times,
                      cudaStream_t s, std::string* err);

}  // namespace line
