// Walk sampler (Algorithms 2-3, the local walk of one partition): the
// positive pair of sample t is pair t mod P of walk t / P, P = L W - W (W-1)/2.
//
// Walk wk: nodes[0], nodes[1] = the arc drawn by weight with the words of
// draw (wk, call 0) in domain 8 (the edge alias table).  Step i = 1 .. L-1
// moves from x = nodes[i] to the out-neighbour picked by words (w0, w1) of
// draw (wk, call i): u = ((w1:w0) >> 11) 2^-53, target = u cw[hi-1] (FP64),
// the first arc e of x with cw[e] > target (the last arc if none), cw the
// running FP64 sum of x's arc weights in arc order.  A node without out-arcs
// steps back to nodes[i-1].  Pairs of a walk: (nodes[i], nodes[i+k]),
// i = 0 .. L-1, k = 1 .. W, i + k <= L, in (i, k) order.  With reuse r (a
// single-device form of the Reuse-Spill variant of §IV-C) each walk's pairs
// serve r passes in a row: sample t takes pair t mod P of walk t / (r P).
//
// One warp per walk: the L steps are sequential, each a row_ptr lookup and a
// lane-parallel search of cw.  A node of at most 32 arcs takes one round of
// loads (every arc's running sum and head, then a ballot); larger ones a
// search of 32 probes per round.  The nodes stay in shared memory while the
// warp writes the pairs of the samples in range.
#include <algorithm>

#include "line_internal.cuh"

namespace line {
namespace {

constexpr uint32_t kWalkDomain = 8u;
constexpr int kWalkWarps = 4;

// row_ptr[v] = first arc of v (src sorted), row_ptr[n] = n_arcs.  Arc e in
// [0, m] fills the nodes between src[e-1] and src[e] (src[m] read as n).
__global__ void k_row_ptr(const int32_t* __restrict__ src, int64_t n_arcs, int64_t n_nodes,
                          int64_t* __restrict__ row_ptr) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e <= n_arcs; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t hi = e < n_arcs ? (int64_t)src[e] : n_nodes;
        const int64_t lo = e > 0 ? (int64_t)src[e - 1] + 1 : 0;
        for (int64_t v = lo; v <= hi; ++v) row_ptr[v] = e;
    }
}

// cw[e]: running sum of the weights of src[e]'s arcs up to e, left to right
// in FP64 (one thread per node, so the rounding order is the arc order).
__global__ void k_cumw(const int64_t* __restrict__ row_ptr, const float* __restrict__ w, int64_t n_nodes,
                       double* __restrict__ cw) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_nodes; v += (int64_t)gridDim.x * blockDim.x) {
        double run = 0.0;
        for (int64_t e = row_ptr[v], hi = row_ptr[v + 1]; e < hi; ++e) {
            run += w ? (double)w[e] : 1.0;
            cw[e] = run;
        }
    }
}

// (i, k) of pair q of a walk: the first L-W+1 nodes own W pairs each, the
// last W-1 nodes W-1, W-2, ..., 1.
__device__ __forceinline__ void pair_of(uint32_t q, int L, int W, int* i, int* k) {
    const uint32_t full = (uint32_t)(L - W + 1) * (uint32_t)W;
    if (q < full) {
        *i = (int)(q / (uint32_t)W);
        *k = (int)(q % (uint32_t)W) + 1;
        return;
    }
    q -= full;
    int ii = L - W + 1;
    uint32_t n = (uint32_t)W - 1u;
    while (q >= n) {
        q -= n;
        --n;
        ++ii;
    }
    *i = ii;
    *k = (int)q + 1;
}

// The first arc of [lo, hi) with cw > target, or hi; called by a full warp
// with warp-uniform arguments.
__device__ __forceinline__ int64_t first_above(const double* __restrict__ cw, int64_t lo, int64_t hi, double target,
                                               int lane) {
    int64_t a = lo, b = hi;  // cw[e] <= target for e < a; b is hi or an arc above the target
    while (b - a > 32) {
        const int64_t step = (b - a + 31) / 32;
        const int64_t pos = min(a + (int64_t)(lane + 1) * step - 1, b - 1);
        const unsigned m = __ballot_sync(0xFFFFFFFFu, __ldg(cw + pos) > target);
        if (m == 0) {
            a = b;  // probe 31 sits at b - 1
        } else {
            const int j = __ffs(m) - 1;
            const int64_t pj = min(a + (int64_t)(j + 1) * step - 1, b - 1);
            const int64_t pprev = j > 0 ? min(a + (int64_t)j * step - 1, b - 1) : a - 1;
            b = pj;
            a = pprev + 1;
        }
    }
    const int64_t e = a + lane;
    const unsigned m = __ballot_sync(0xFFFFFFFFu, e < b && __ldg(cw + e) > target);
    return m ? a + (__ffs(m) - 1) : b;
}

__global__ void __launch_bounds__(kWalkWarps * 32) k_walk_pairs(WalkParams p) {
    extern __shared__ int32_t s_nodes[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t* nodes = s_nodes + warp * (p.L + 1);
    const uint64_t P = p.P, RP = p.P * (uint64_t)p.reuse;
    const uint64_t w_first = p.t0 / RP, w_last = (p.t0 + (uint64_t)p.count - 1) / RP;
    for (uint64_t wk = w_first + (uint64_t)blockIdx.x * kWalkWarps + warp; wk <= w_last;
         wk += (uint64_t)gridDim.x * kWalkWarps) {
        int32_t prev, x;
        {
            const uint4 w = draw_words(p.seed, kWalkDomain, wk, 0u);
            const uint32_t e = alias_pick(p.edge_tab, (uint64_t)p.n_arcs, w);
            prev = __ldg(p.src + e);
            x = __ldg(p.dst + e);
        }
        if (lane == 0) {
            nodes[0] = prev;
            nodes[1] = x;
        }
        for (int i = 1; i < p.L; ++i) {
            const int64_t lo = __ldg(p.row_ptr + x), hi = __ldg(p.row_ptr + x + 1);
            int32_t next = prev;  // a dead end steps back
            if (lo < hi) {
                const uint4 w = draw_words(p.seed, kWalkDomain, wk, (uint32_t)i);
                const uint64_t r = (((uint64_t)w.y << 32) | (uint64_t)w.x) >> 11;
                const double u = (double)r * 0x1p-53;
                const int64_t deg = hi - lo;
                if (deg <= 32) {
                    // one round of loads: every arc's running sum and head
                    const bool in = lane < deg;
                    const double cwl = in ? __ldg(p.cw + lo + lane) : 0.0;
                    const int32_t dl = in ? __ldg(p.dst + lo + lane) : 0;
                    const double target = u * __shfl_sync(0xFFFFFFFFu, cwl, (int)deg - 1);
                    const unsigned m = __ballot_sync(0xFFFFFFFFu, in && cwl > target);
                    next = __shfl_sync(0xFFFFFFFFu, dl, m ? __ffs(m) - 1 : (int)deg - 1);
                } else {
                    const double target = u * __ldg(p.cw + hi - 1);
                    const int64_t f = first_above(p.cw, lo, hi, target, lane);
                    next = __ldg(p.dst + (f < hi ? f : hi - 1));
                }
            }
            prev = x;
            x = next;
            if (lane == 0) nodes[i + 1] = x;
        }
        __syncwarp();
        const uint64_t s_begin = max(wk * RP, p.t0), s_end = min((wk + 1) * RP, p.t0 + (uint64_t)p.count);
        for (uint64_t t = s_begin + lane; t < s_end; t += 32) {
            int i, k;
            pair_of((uint32_t)((t - wk * RP) % P), p.L, p.W, &i, &k);
            const int32_t u = nodes[i], v = nodes[i + k];
            const uint64_t s = t - p.t0;
            p.rec[s * p.R] = u;
            p.rec[s * p.R + 1] = v;
            if (p.items) {
                const uint64_t lowbits = (uint32_t)s << p.slot_bits;  // s < 2^26 within a chunk
                p.items[s * p.R] = ((uint64_t)(uint32_t)u << 32) | lowbits;
                p.items[s * p.R + 1] = ((uint64_t)((uint32_t)v + p.ctx_off) << 32) | lowbits | 1u;
            }
        }
        __syncwarp();  // the nodes are rewritten by the warp's next walk
    }
}

}  // namespace

size_t walk_smem_bytes(int L) { return sizeof(int32_t) * (size_t)kWalkWarps * (size_t)(L + 1); }

cudaError_t row_offsets(int64_t n_nodes, int64_t n_arcs, const int32_t* src, int64_t* row_ptr, cudaStream_t s) {
    const unsigned g = (unsigned)std::min<int64_t>((n_arcs + 1 + 255) / 256, 152 * 32);
    k_row_ptr<<<g, 256, 0, s>>>(src, n_arcs, n_nodes, row_ptr);
    return cudaGetLastError();
}

cudaError_t walk_cumw(int64_t n_nodes, const int64_t* row_ptr, const float* w, double* cw, cudaStream_t s) {
    const unsigned g = (unsigned)std::min<int64_t>((n_nodes + 127) / 128, 152 * 32);
    k_cumw<<<g, 128, 0, s>>>(row_ptr, w, n_nodes, cw);
    return cudaGetLastError();
}

cudaError_t walk_pairs(const WalkParams& p, cudaStream_t s) {
    if (p.count <= 0) return cudaSuccess;
    const uint64_t RP = p.P * (uint64_t)p.reuse;
    const uint64_t n_walks = (p.t0 + (uint64_t)p.count - 1) / RP - p.t0 / RP + 1;
    const unsigned g = (unsigned)std::min<uint64_t>((n_walks + kWalkWarps - 1) / kWalkWarps, 152 * 16);
    k_walk_pairs<<<g, kWalkWarps * 32, walk_smem_bytes(p.L), s>>>(p);
    return cudaGetLastError();
}

}  // namespace line
