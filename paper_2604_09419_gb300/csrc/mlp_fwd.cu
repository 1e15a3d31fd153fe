// Forward products of the warm-start MLP with BF16 activations (see
// mlp_fwd.cuh for the operation): one persistent CTA per SM loops over
// 128-row tiles of A.
//
//   warp 0     (one lane) copies the weights' hi and lo tiles into shared
//              memory once (one bulk copy), then streams A through a ring
//              of stages: per tile, ceil(K/64) TMA loads of 128 rows x 64
//              BF16 (128-byte rows, 128-byte swizzle); rows beyond M and
//              columns beyond K arrive as zeros;
//   warp 1     allocates 2N tensor-memory columns (two accumulators) and
//              issues, per stage, two tcgen05.mma kind::f16 (A x W_hi^T,
//              A x W_lo^T) for every 16 columns of K inside [0, K), into
//              the tile's accumulator; a commit frees the stage when its
//              products are done, another marks the accumulator full;
//   warps 2-17 the epilogue: warp w reads rows 32 (w % 4) .. + 31 of the
//              accumulator (its tensor-memory lanes), one quarter of the
//              columns, 16 at a time (tcgen05.ld), adds the bias, applies
//              GELU, writes the 32 x 16 block into its staging buffer in the
//              swizzled layout of the output's tensor map, and one lane
//              stores the block with a TMA tensor store (rows beyond M
//              clipped); then it releases the accumulator, so that the
//              products of tile i+1 run while tile i is written out.  Four
//              epilogue warps per scheduler keep the GELU's instruction
//              stream issuing.
//
// Every wait is bounded: a wait that runs out records DEV_ERR_TIMEOUT and
// raises the CTA's abort flag, on which the other roles stop; before the
// CTA exits, the copy lane waits (bounded) for its own copies in flight and
// the product lane for its own products, and warp 1 frees the tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "bulk.cuh"
#include "line_internal.cuh"
#include "mlp_fwd.cuh"
#include "mlp_math.cuh"

namespace line {

namespace {

constexpr int kFM = 128;                                 // rows of a tile (the products' M)
constexpr int kFKS = 64;                                 // K per stage: one 128-byte row of BF16
constexpr uint32_t kFStageBytes = kFM * kFKS * 2;        // 16 KB
constexpr int kFMaxStages = 4;
constexpr int kFEpiWarps = 16;
constexpr int kFChunk = 16;  // accumulator columns per tcgen05.ld and per stored block
constexpr int kFThreads = 32 * (2 + kFEpiWarps);         // copy warp, product warp, epilogue warps
constexpr size_t kFSmemLimit = 226 * 1024;  // dynamic shared memory of one CTA (227 KB less the static part)
constexpr int64_t kFWaitLimit = int64_t(1) << 24;        // polls of one mbarrier wait

// What the epilogue makes of the sums C:
//   kModeOut     Y = C (FP32), by TMA stores;
//   kModeHidden  A1 = C + b (FP32, optional) and H = GELU(C + b) (BF16, TMA);
//   kModeDact    dA = C GELU'(A1) (FP32) and its BF16 hi/lo pair, stored
//                directly; A enters as its hi/lo pair (two A streams).
enum { kModeOut = 0, kModeHidden = 1, kModeDact = 2 };

struct FwdArgs {
    int M, N, K, n_tiles, stages;
    int mode;
    int nA;                   // A matrices per stage: 1, or 2 (hi, lo) in kModeDact
    const __nv_bfloat16* Wt;  // W_hi then W_lo, core-matrix layout
    const float* bias;        // kModeHidden: [N], 16-byte aligned
    float* A1;                // kModeHidden, nullable: [M][N] sums + bias
    const float* A1in;        // kModeDact: [M][N] the pre-activations
    float* dA;                // kModeDact: [M][N]
    __nv_bfloat16* dA_hl;     // kModeDact: [2][M][N] hi, lo
    uint32_t* status;
};

// Staging buffer of one epilogue warp: a 32 x 16 block of the output (BF16
// rows of 32 bytes for H, FP32 rows of 64 bytes for Y; none for dA).
constexpr uint32_t out_block_bytes(int mode) { return mode == kModeHidden ? 32 * 32 : mode == kModeOut ? 32 * 64 : 0; }

size_t w_bytes(int N, int K) { return fwd_w16_elems(N, K) * sizeof(__nv_bfloat16); }

int stages_for(int N, int K, int mode, int nA) {
    // 1024: room to align the stages
    const size_t fixed = 1024 + w_bytes(N, K) + (size_t)kFEpiWarps * out_block_bytes(mode);
    if (fixed >= kFSmemLimit) return 0;
    return (int)std::min<size_t>(kFMaxStages, (kFSmemLimit - fixed) / ((size_t)nA * kFStageBytes));
}

size_t smem_bytes(int N, int K, int stages, int mode, int nA) {
    return 1024 + (size_t)stages * nA * kFStageBytes + w_bytes(N, K) + (size_t)kFEpiWarps * out_block_bytes(mode);
}

// Shared-memory descriptor of an A stage: start >> 4; leading offset unused
// for a swizzled K-major operand (1); 1024 bytes between groups of 8 rows;
// version 1 at bits 46-47; 128-byte swizzle (2) at bits 61-63.  A step of 16
// values along K inside the 128-byte row adds 32 bytes to the start.
__device__ __forceinline__ uint64_t desc_a(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Descriptor of a weight tile without swizzle: core matrices (8 rows x 16
// bytes) 128 bytes apart along K, groups of 8 rows `sbo` bytes apart.
__device__ __forceinline__ uint64_t desc_w(uint32_t addr, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D = F32 (bits 4-5), A = B = BF16
// (bits 7-9, 10-12), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kFM >> 4) << 24);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// TMA tensor store of the block at src (laid out as the map's box, swizzled
// as the map says) to columns x.., rows y.. of the map's tensor.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_addr(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// This thread's bulk stores have read their shared-memory sources.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// This thread's bulk stores are complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Arrives on `bar` once every earlier tcgen05.mma of this thread is done.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 tensor-memory lanes (one row per lane).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Wait for the phase of `bar` of the given parity.  False when another role
// aborted, or when the wait ran out (then this role aborts the CTA).
__device__ __forceinline__ bool fwd_wait(uint64_t* bar, uint32_t parity, volatile uint32_t* abort_flag,
                                         uint32_t* status) {
    for (int64_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (it > kFWaitLimit) {
            *abort_flag = 1u;
            atomicOr(status, DEV_ERR_TIMEOUT);
            return false;
        }
    }
}

// The same wait regardless of the abort flag, for a role's own copies or
// products before the CTA exits (bounded as well).
__device__ __forceinline__ void fwd_drain(uint64_t* bar, uint32_t parity) {
    for (int64_t it = 0; it <= kFWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__global__ void __launch_bounds__(kFThreads, 1) k_mlp_fwd_tc(const __grid_constant__ CUtensorMap tmA,
                                                             const __grid_constant__ CUtensorMap tmA2,
                                                             const __grid_constant__ CUtensorMap tmO, FwdArgs a) {
    extern __shared__ unsigned char fwd_raw[];
    __shared__ __align__(8) uint64_t full[kFMaxStages], empty[kFMaxStages], tfull[2], tempty[2], wbar, fin;
    __shared__ uint32_t tmem_base;
    __shared__ uint32_t abort_word;
    volatile uint32_t* abort_flag = &abort_word;
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(fwd_raw) + 1023) & ~(uintptr_t)1023);
    const int S = a.stages, N = a.N, K = a.K;
    const uint32_t sbytes = (uint32_t)a.nA * kFStageBytes;  // a stage: A (or A_hi, A_lo), 16 KB each
    unsigned char* sA = base;                                // S stages
    __nv_bfloat16* sW = reinterpret_cast<__nv_bfloat16*>(base + (size_t)S * sbytes);  // W_hi, W_lo
    // the epilogue warps' staging blocks (1024-byte aligned: N K 4 is a multiple of 4096)
    const uint32_t wbytes = (uint32_t)(2 * (size_t)N * K * sizeof(__nv_bfloat16));
    unsigned char* sOut = base + (size_t)S * sbytes + (size_t)wbytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nks = (K + kFKS - 1) / kFKS;
    uint32_t cols = 32;
    while (cols < 2u * (uint32_t)N) cols <<= 1;
    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], kFEpiWarps);
        }
        mbar_init(&wbar, 1);
        mbar_init(&fin, 1);
        abort_word = 0u;
        mbar_init_fence();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            mbar_arrive_expect_tx(&wbar, wbytes);
            bulk_load(sW, a.Wt, wbytes, &wbar);
            uint32_t g = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < a.n_tiles; t += gridDim.x) {
                for (int ks = 0; ks < nks; ++ks) {
                    const uint32_t st = g % (uint32_t)S, j = g / (uint32_t)S;
                    if (!fwd_wait(&empty[st], (j & 1u) ^ 1u, abort_flag, a.status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[st], sbytes);
                    tma_load_2d(sA + (size_t)st * sbytes, &tmA, ks * kFKS, t * kFM, &full[st]);
                    if (a.nA == 2) tma_load_2d(sA + (size_t)st * sbytes + kFStageBytes, &tmA2, ks * kFKS, t * kFM, &full[st]);
                    ++g;
                }
            }
            // this lane's copies in flight: the weights, and after an abort
            // the last S stage loads (earlier ones were consumed)
            fwd_drain(&wbar, 0u);
            if (!ok) {
                for (uint32_t i = 0; i < (uint32_t)S && i < g; ++i) {
                    const uint32_t gg = g - 1 - i;
                    fwd_drain(&full[gg % (uint32_t)S], (gg / (uint32_t)S) & 1u);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = fwd_wait(&wbar, 0u, abort_flag, a.status);
            tc_fence_after();
            const uint32_t w_hi = smem_addr(sW), w_lo = w_hi + (uint32_t)((size_t)N * K * sizeof(__nv_bfloat16));
            const uint32_t sbo = (uint32_t)K * 16u;  // 8 rows of K BF16
            const uint32_t idesc = idesc_bf16(N);
            uint32_t g = 0, i = 0;
            for (int t = blockIdx.x; ok && t < a.n_tiles; t += gridDim.x, ++i) {
                const uint32_t acc = i & 1u, u = i >> 1;
                if (!fwd_wait(&tempty[acc], (u & 1u) ^ 1u, abort_flag, a.status)) break;
                tc_fence_after();
                const uint32_t d = tmem + acc * (uint32_t)N;
                for (int ks = 0; ks < nks; ++ks, ++g) {
                    const uint32_t st = g % (uint32_t)S, j = g / (uint32_t)S;
                    if (!fwd_wait(&full[st], j & 1u, abort_flag, a.status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_addr(sA + (size_t)st * sbytes);
#pragma unroll
                    for (int kk = 0; kk < kFKS / 16; ++kk) {
                        const int k = ks * kFKS + kk * 16;
                        if (k >= K) break;
                        const uint64_t da = desc_a(sa + (uint32_t)kk * 32u);
                        const uint32_t wo = (uint32_t)(k >> 3) * 128u;
                        tc_mma(d, da, desc_w(w_hi + wo, sbo), idesc, (ks | kk) ? 1u : 0u);
                        tc_mma(d, da, desc_w(w_lo + wo, sbo), idesc, 1u);
                        // A_lo W_hi; A_lo W_lo, about 2^-18 of the product, is left
                        // out, as the weights' own truncation at about 2^-17 is
                        if (a.nA == 2) tc_mma(d, desc_a(sa + kFStageBytes + (uint32_t)kk * 32u), desc_w(w_hi + wo, sbo), idesc, 1u);
                    }
                    tc_commit(&empty[st]);  // the stage is free once these products are done
                }
                if (!ok) break;
                tc_commit(&tfull[acc]);
            }
            // every product of this lane done before the CTA exits
            tc_commit(&fin);
            fwd_drain(&fin, 0u);
        }
        __syncwarp();
    } else {
        const int e = warp - 2, q = warp & 3, h = e >> 2;
        const int quarter = N / 4;
        const int mode = a.mode;
        const bool hid = mode == kModeHidden;
        unsigned char* blk = sOut + (size_t)e * out_block_bytes(mode);
        const uint32_t so = smem_addr(blk);
        uint32_t i = 0;
        for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x, ++i) {
            const uint32_t acc = i & 1u, u = i >> 1;
            const int row0 = t * kFM + q * 32, row = row0 + lane;
            const int c_end = (h + 1) * quarter;
            // dL/da: the pre-activations of this warp's first 16 columns are
            // loaded before the products are waited for, and those of the
            // next 16 columns while the current ones are worked on
            float4 a1_next[4];
            if (mode == kModeDact && row < a.M) {
                const float4* ap = reinterpret_cast<const float4*>(a.A1in + (size_t)row * N + h * quarter);
#pragma unroll
                for (int j = 0; j < 4; ++j) a1_next[j] = __ldg(ap + j);
            }
            const bool ok = fwd_wait(&tfull[acc], u & 1u, abort_flag, a.status);
            if (!__all_sync(0xFFFFFFFFu, ok)) break;
            tc_fence_after();
            for (int c0 = h * quarter; c0 < c_end; c0 += kFChunk) {
                uint32_t r[16];
                tc_ld16(tmem + ((uint32_t)(q * 32) << 16) + acc * (uint32_t)N + (uint32_t)c0, r);
                if (mode == kModeDact) {
                    // dA = C GELU'(A1), FP32 and its BF16 hi/lo pair, this row's 16 columns
                    if (row < a.M) {
                        const size_t o = (size_t)row * N + c0;
                        float4 a1_cur[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) a1_cur[j] = a1_next[j];
                        if (c0 + kFChunk < c_end) {
                            const float4* ap = reinterpret_cast<const float4*>(a.A1in + o + kFChunk);
#pragma unroll
                            for (int j = 0; j < 4; ++j) a1_next[j] = __ldg(ap + j);
                        }
                        float v[16];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float4 a1 = a1_cur[j];
                            const float2 g0 = __fmul2_rn(make_float2(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1])),
                                                         gelu_grad_fast2(make_float2(a1.x, a1.y)));
                            const float2 g1 = __fmul2_rn(make_float2(__uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3])),
                                                         gelu_grad_fast2(make_float2(a1.z, a1.w)));
                            v[4 * j] = g0.x;
                            v[4 * j + 1] = g0.y;
                            v[4 * j + 2] = g1.x;
                            v[4 * j + 3] = g1.y;
                        }
                        float4* dp = reinterpret_cast<float4*>(a.dA + o);
#pragma unroll
                        for (int j = 0; j < 4; ++j) dp[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                        float hi[16], lo[16];
#pragma unroll
                        for (int j = 0; j < 16; j += 2) {
                            hi[j] = __bfloat162float(__float2bfloat16_rn(v[j]));
                            hi[j + 1] = __bfloat162float(__float2bfloat16_rn(v[j + 1]));
                            const float2 l = __fadd2_rn(make_float2(v[j], v[j + 1]), make_float2(-hi[j], -hi[j + 1]));
                            lo[j] = l.x;
                            lo[j + 1] = l.y;
                        }
                        uint4* hp = reinterpret_cast<uint4*>(a.dA_hl + o);
                        uint4* lp = reinterpret_cast<uint4*>(a.dA_hl + (size_t)a.M * N + o);
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            hp[j] = make_uint4(pack_bf16x2(hi[8 * j], hi[8 * j + 1]), pack_bf16x2(hi[8 * j + 2], hi[8 * j + 3]),
                                               pack_bf16x2(hi[8 * j + 4], hi[8 * j + 5]), pack_bf16x2(hi[8 * j + 6], hi[8 * j + 7]));
                            lp[j] = make_uint4(pack_bf16x2(lo[8 * j], lo[8 * j + 1]), pack_bf16x2(lo[8 * j + 2], lo[8 * j + 3]),
                                               pack_bf16x2(lo[8 * j + 4], lo[8 * j + 5]), pack_bf16x2(lo[8 * j + 6], lo[8 * j + 7]));
                        }
                    }
                    continue;
                }
                // the block's previous store has read the staging buffer
                if (lane == 0) bulk_wait_read();
                __syncwarp();
                if (hid) {
                    float v[16];
                    const float4* bp = reinterpret_cast<const float4*>(a.bias + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float4 b = __ldg(bp + j);
                        const float2 s0 = __fadd2_rn(make_float2(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1])),
                                                     make_float2(b.x, b.y));
                        const float2 s1 = __fadd2_rn(make_float2(__uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3])),
                                                     make_float2(b.z, b.w));
                        v[4 * j] = s0.x;
                        v[4 * j + 1] = s0.y;
                        v[4 * j + 2] = s1.x;
                        v[4 * j + 3] = s1.y;
                    }
                    if (a.A1 && row < a.M) {
                        float4* p = reinterpret_cast<float4*>(a.A1 + (size_t)row * N + c0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) p[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    }
                    // row `lane` of the block: 2 pieces of 16 bytes, piece j at
                    // j ^ ((lane >> 2) & 1) (the map's 32-byte swizzle)
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        uint32_t w[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float2 gq = gelu_bf16out2(make_float2(v[8 * j + 2 * q], v[8 * j + 2 * q + 1]));
                            w[q] = pack_bf16x2(gq.x, gq.y);
                        }
                        st_shared_v4(so + (uint32_t)lane * 32u + ((uint32_t)(j ^ ((lane >> 2) & 1)) << 4), w[0], w[1],
                                     w[2], w[3]);
                    }
                } else {
                    // 4 pieces of 16 bytes, piece j at j ^ ((lane >> 1) & 3) (64-byte swizzle)
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        st_shared_v4(so + (uint32_t)lane * 64u + ((uint32_t)(j ^ ((lane >> 1) & 3)) << 4), r[4 * j],
                                     r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
                }
                fence_proxy_async_smem();  // the tensor store reads the block through the async proxy
                __syncwarp();
                if (lane == 0) {
                    tma_store_2d(&tmO, c0, row0, blk);
                    bulk_commit();
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
        }
        if (lane == 0) bulk_wait_all();  // the stores are done before the CTA's shared memory goes
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
    }
}


// ---------------------------------------------------------------------------
// Weight gradients with BF16 activations: G[m][n] = sum_k A[k][m] B[k][n]
// over the batch k, for A = dL/dy or dL/da (FP32, given as its BF16 hi/lo
// pair) and B = h or x (BF16).  A and B are row-major over the batch, so
// both enter the products M/N-major: TMA boxes of 64 columns x 64 batch rows
// (128-byte rows, 128-byte swizzle), consecutive 64-column boxes 8 KB apart.
// Split over K: CTA (z, y) takes batch rows [z Ks, (z+1) Ks) and the 128
// rows y*128 .. of G, and writes its partial sums to part[z] (summed in z
// order by the caller).  Warp 0 copies, warp 1 issues the products
// (A_hi B, then A_lo B, per 16 batch rows), warps 2-5 write the partial.
// ---------------------------------------------------------------------------
constexpr int kWK = 64;                     // batch rows per stage
constexpr uint32_t kWBox = 64 * kWK * 2;    // one 64-column box of a stage: 8 KB
constexpr int kWStages = 3;
constexpr int kWThreads = 32 * 6;

struct WgradArgs {
    int M, N, K, Ks, nkb;  // nkb: 64-column boxes of B
    float* part;           // [S][M][N]
    uint32_t* status;
};

__host__ __device__ constexpr uint32_t w_stage_bytes(int nkb) { return 4 * kWBox + (uint32_t)nkb * kWBox; }

// Descriptor of an M/N-major operand in a stage: start >> 4; 8 KB between
// 64-column boxes (leading); 1024 bytes between groups of 8 batch rows
// (stride); version 1; 128-byte swizzle.  16 batch rows further on is 2 KB.
__device__ __forceinline__ uint64_t desc_mn(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(kWBox >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// kind::f16, D = F32, A = B = BF16, both M/N-major (bits 15, 16).
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kFM >> 4) << 24);
}

__global__ void __launch_bounds__(kWThreads, 1)
    k_mlp_wgrad_tc(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                   const __grid_constant__ CUtensorMap tmB, WgradArgs a) {
    extern __shared__ unsigned char w_raw[];
    __shared__ __align__(8) uint64_t full[kWStages], empty[kWStages], tfull, fin;
    __shared__ uint32_t tmem_base;
    __shared__ uint32_t abort_word;
    volatile uint32_t* abort_flag = &abort_word;
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(w_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = a.N;
    const uint32_t sbytes = w_stage_bytes(a.nkb);
    const int z = blockIdx.x, m0 = blockIdx.y * kFM;
    const int k0 = z * a.Ks, k1 = min(a.K, k0 + a.Ks);
    const int nst = (k1 - k0 + kWK - 1) / kWK;
    uint32_t cols = 32;
    while (cols < (uint32_t)N) cols <<= 1;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kWStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&tfull, 1);
        mbar_init(&fin, 1);
        abort_word = 0u;
        mbar_init_fence();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            for (int i = 0; i < nst; ++i, ++g) {
                const uint32_t st = g % kWStages, j = g / kWStages;
                if (!fwd_wait(&empty[st], (j & 1u) ^ 1u, abort_flag, a.status)) {
                    ok = false;
                    break;
                }
                unsigned char* sp = base + (size_t)st * sbytes;
                const int kr = k0 + i * kWK;
                mbar_arrive_expect_tx(&full[st], sbytes);
                // stage: A_hi (2 boxes), A_lo (2 boxes), B (nkb boxes)
                tma_load_2d(sp, &tmAh, m0, kr, &full[st]);
                tma_load_2d(sp + kWBox, &tmAh, m0 + 64, kr, &full[st]);
                tma_load_2d(sp + 2 * kWBox, &tmAl, m0, kr, &full[st]);
                tma_load_2d(sp + 3 * kWBox, &tmAl, m0 + 64, kr, &full[st]);
                for (int b = 0; b < a.nkb; ++b) tma_load_2d(sp + (4 + b) * kWBox, &tmB, 64 * b, kr, &full[st]);
            }
            if (!ok) {
                for (uint32_t i = 0; i < (uint32_t)kWStages && i < g; ++i) {
                    const uint32_t gg = g - 1 - i;
                    fwd_drain(&full[gg % kWStages], (gg / kWStages) & 1u);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_mn(N);
            bool ok = true;
            for (int i = 0; i < nst; ++i) {
                const uint32_t st = (uint32_t)i % kWStages, j = (uint32_t)i / kWStages;
                if (!fwd_wait(&full[st], j & 1u, abort_flag, a.status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sp = smem_addr(base + (size_t)st * sbytes);
#pragma unroll
                for (int kk = 0; kk < kWK / 16; ++kk) {
                    const uint32_t off = (uint32_t)kk * 2048u;
                    const uint64_t db = desc_mn(sp + 4 * kWBox + off);
                    tc_mma(tmem, desc_mn(sp + off), db, idesc, (i | kk) ? 1u : 0u);
                    tc_mma(tmem, desc_mn(sp + 2 * kWBox + off), db, idesc, 1u);
                }
                tc_commit(&empty[st]);
            }
            if (ok && nst > 0) tc_commit(&tfull);
            tc_commit(&fin);
            fwd_drain(&fin, 0u);
        }
        __syncwarp();
    } else {
        const int q = warp & 3;
        bool ok = nst > 0 && fwd_wait(&tfull, 0u, abort_flag, a.status);
        ok = __all_sync(0xFFFFFFFFu, ok);
        if (ok) {
            tc_fence_after();
            const int row = m0 + q * 32 + lane;
            float* out = a.part + ((size_t)z * a.M + row) * N;
            for (int c0 = 0; c0 < N; c0 += kFChunk) {
                uint32_t r[16];
                tc_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
                if (row < a.M) {
                    float4* p = reinterpret_cast<float4*>(out + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        p[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                           __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
                }
            }
        } else if (nst == 0 && lane == 0) {
            // an empty slice: zero partial sums
            for (int rr = 0; rr < 32; ++rr) {
                const int row = m0 + q * 32 + rr;
                if (row < a.M)
                    for (int c = 0; c < N; ++c) a.part[((size_t)z * a.M + row) * N + c] = 0.0f;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
    }
}

// W -> hi/lo BF16 tiles (see fwd_tile_weights); TRANS: W is stored K x N
// (row-major), its transpose is tiled.
template <bool TRANS>
__global__ void k_tile_w16(const float* __restrict__ W, int N, int K, __nv_bfloat16* __restrict__ Wt) {
    const int64_t total = (int64_t)N * K;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(i / K), k = (int)(i % K);
        const float w = TRANS ? W[(int64_t)k * N + n] : W[i];
        const __nv_bfloat16 hi = __float2bfloat16_rn(w);
        const __nv_bfloat16 lo = __float2bfloat16_rn(w - __bfloat162float(hi));  // w - hi is exact in FP32
        const int64_t o = (int64_t)(n >> 3) * (K * 8) + (k >> 3) * 64 + (n & 7) * 8 + (k & 7);
        Wt[o] = hi;
        Wt[total + o] = lo;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

}  // namespace

bool fwd_tc_supported(int N, int K) {
    // (the output layer's staging is the larger: both layers fit when it does)
    return N >= 64 && N <= 256 && N % (4 * kFChunk) == 0 && K >= 16 && K % 16 == 0 &&
           stages_for(N, K, kModeOut, 1) >= 2;
}

cudaError_t fwd_tile_weights(const float* W, int N, int K, __nv_bfloat16* Wt, cudaStream_t s) {
    const int64_t total = (int64_t)N * K;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 1024);
    k_tile_w16<false><<<blocks, 256, 0, s>>>(W, N, K, Wt);
    return cudaGetLastError();
}

namespace {

// One launch of k_mlp_fwd_tc in `mode` (see kModeOut ...).
cudaError_t launch_fwd(int mode, int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* A_lo,
                       const __nv_bfloat16* Wt, const float* bias, float* A1, const float* A1in, __nv_bfloat16* H,
                       float* Y, float* dA, __nv_bfloat16* dA_hl, uint32_t* status, cudaStream_t s) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = encode_tiled();
    if (!encode) return cudaErrorNotSupported;
    const int nA = A_lo ? 2 : 1;
    const cuuint32_t elem_strides[2] = {1, 1};
    // A (and A_lo): K columns (inner) x M rows, row pitch 2K bytes; boxes of 64 x 128
    auto a_map = [&](CUtensorMap* map, const __nv_bfloat16* p) {
        const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)M};
        const cuuint64_t strides[1] = {(cuuint64_t)K * sizeof(__nv_bfloat16)};
        const cuuint32_t box[2] = {(cuuint32_t)kFKS, (cuuint32_t)kFM};
        return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(p), dims, strides, box,
                      elem_strides, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    CUtensorMap map, map2;
    if (!a_map(&map, A) || !a_map(&map2, A_lo ? A_lo : A)) return cudaErrorInvalidValue;
    // the output of kModeHidden (H: BF16) or kModeOut (Y: FP32): N columns x
    // M rows, boxes of 16 x 32, swizzled over the box's row (32 or 64 bytes);
    // kModeDact stores directly and takes the A map as a placeholder
    CUtensorMap omap = map;
    if (mode != kModeDact) {
        const bool hidden = mode == kModeHidden;
        const size_t esz = hidden ? sizeof(__nv_bfloat16) : sizeof(float);
        const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)M};
        const cuuint64_t strides[1] = {(cuuint64_t)N * esz};
        const cuuint32_t box[2] = {(cuuint32_t)kFChunk, 32};
        if (encode(&omap, hidden ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                   hidden ? (void*)H : (void*)Y, dims, strides, box, elem_strides, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   hidden ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int stages = stages_for(N, K, mode, nA);
    if (stages < 2) return cudaErrorInvalidValue;
    const size_t smem = smem_bytes(N, K, stages, mode, nA);
    {
        // the kernel's dynamic shared-memory limit, raised per device to the
        // largest launch so far
        static std::mutex mu;
        static size_t granted[64] = {};
        std::lock_guard<std::mutex> lock(mu);
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (granted[dev] < smem) {
            e = cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            granted[dev] = smem;
        }
    }
    FwdArgs a;
    a.M = M;
    a.N = N;
    a.K = K;
    a.n_tiles = (M + kFM - 1) / kFM;
    a.stages = stages;
    a.mode = mode;
    a.nA = nA;
    a.Wt = Wt;
    a.bias = bias;
    a.A1 = mode == kModeHidden ? A1 : nullptr;
    a.A1in = A1in;
    a.dA = dA;
    a.dA_hl = dA_hl;
    a.status = status;
    const int grid = std::min(a.n_tiles, sms);
    k_mlp_fwd_tc<<<grid, kFThreads, smem, s>>>(map, map2, omap, a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t fwd_tc(int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* Wt, const float* bias, float* A1,
                   __nv_bfloat16* H, float* Y, uint32_t* status, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    const bool hidden = H != nullptr;
    if (!fwd_tc_supported(N, K) || (hidden ? bias == nullptr || (reinterpret_cast<uintptr_t>(bias) & 15) : Y == nullptr))
        return cudaErrorInvalidValue;
    return launch_fwd(hidden ? kModeHidden : kModeOut, M, N, K, A, nullptr, Wt, bias, A1, nullptr, H, Y, nullptr,
                      nullptr, status, s);
}

bool dact_tc_supported(int N, int K) {
    return N >= 64 && N <= 256 && N % (4 * kFChunk) == 0 && K >= 16 && K % 16 == 0 &&
           stages_for(N, K, kModeDact, 2) >= 2;
}

cudaError_t dact_tc(int M, int N, int K, const __nv_bfloat16* A_hi, const __nv_bfloat16* A_lo,
                    const __nv_bfloat16* Wt, const float* A1, float* dA, __nv_bfloat16* dA_hl, uint32_t* status,
                    cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    if (!dact_tc_supported(N, K) || !A_lo || !A1 || !dA || !dA_hl) return cudaErrorInvalidValue;
    return launch_fwd(kModeDact, M, N, K, A_hi, A_lo, Wt, nullptr, nullptr, A1, nullptr, nullptr, dA, dA_hl, status,
                      s);
}

cudaError_t fwd_tile_weights_t(const float* W, int N, int K, __nv_bfloat16* Wt, cudaStream_t s) {
    const int64_t total = (int64_t)N * K;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 1024);
    k_tile_w16<true><<<blocks, 256, 0, s>>>(W, N, K, Wt);
    return cudaGetLastError();
}

bool wgrad_tc_supported(int M, int N) {
    return M >= kFM && M % kFM == 0 && N >= 16 && N <= 256 && N % 16 == 0 &&
           1024 + (size_t)kWStages * w_stage_bytes((N + 63) / 64) <= kFSmemLimit;
}

namespace {
// batch rows per slice: a multiple of 64, at most kWgradMaxSlices slices
int wgrad_rows_per(int K) {
    const int per = (K + kWgradMaxSlices - 1) / kWgradMaxSlices;
    return std::max(kWK, (per + kWK - 1) / kWK * kWK);
}
}  // namespace

int wgrad_slices(int K) { return K <= 0 ? 0 : (K + wgrad_rows_per(K) - 1) / wgrad_rows_per(K); }

cudaError_t wgrad_tc(int M, int N, int K, const __nv_bfloat16* A_hi, const __nv_bfloat16* A_lo,
                     const __nv_bfloat16* B, float* part, uint32_t* status, cudaStream_t s) {
    if (K <= 0) return cudaErrorInvalidValue;
    if (!wgrad_tc_supported(M, N)) return cudaErrorInvalidValue;
    PFN_cuTensorMapEncodeTiled_v12000 encode = encode_tiled();
    if (!encode) return cudaErrorNotSupported;
    const cuuint32_t elem_strides[2] = {1, 1};
    const cuuint32_t box[2] = {64, (cuuint32_t)kWK};
    // row-major over the batch: `cols` columns (inner) x K rows
    auto make = [&](CUtensorMap* map, const __nv_bfloat16* p, int cols) {
        const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)K};
        const cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(__nv_bfloat16)};
        return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(p), dims, strides, box,
                      elem_strides, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    CUtensorMap mah, mal, mb;
    if (!make(&mah, A_hi, M) || !make(&mal, A_lo, M) || !make(&mb, B, N)) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int nkb = (N + 63) / 64;
    const size_t smem = 1024 + (size_t)kWStages * w_stage_bytes(nkb);
    {
        static std::mutex mu;
        static size_t granted[64] = {};
        std::lock_guard<std::mutex> lock(mu);
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (granted[dev] < smem) {
            e = cudaFuncSetAttribute(k_mlp_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            granted[dev] = smem;
        }
    }
    WgradArgs w;
    w.M = M;
    w.N = N;
    w.K = K;
    w.Ks = wgrad_rows_per(K);
    w.nkb = nkb;
    w.part = part;
    w.status = status;
    k_mlp_wgrad_tc<<<dim3((unsigned)wgrad_slices(K), (unsigned)(M / kFM)), kWThreads, smem, s>>>(mah, mal, mb, w);
    return cudaGetLastError();
}

}  // namespace line
