// Row access shared by the training kernels (train.cu, hogwild.cu): the
// lane geometry of a row, FP32/BF16 row loads, and row stores with BF16
// stochastic rounding.
#pragma once

#include "line_internal.cuh"

namespace line {

// ---------------------------------------------------------------------------
// Row geometry: a row of D values is handled by L lanes, E values per lane,
// moved as vectors of 4 values (16 bytes of FP32, 8 bytes of BF16).
// ---------------------------------------------------------------------------
// (host and device share these two: the work-item map of the persistent
// schedule is laid out on the host)
constexpr int geom_vec(int /*dtype*/) { return 4; }
constexpr int geom_lanes(int dim, int dtype) { return dim / geom_vec(dtype) < 32 ? dim / geom_vec(dtype) : 32; }

template <int D, int DT>
struct Geom {
    static constexpr int VEC = geom_vec(DT);
    static constexpr int L = geom_lanes(D, DT);
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
        const uint2* p = reinterpret_cast<const uint2*>(reinterpret_cast<const __nv_bfloat16*>(table) + row * D + lig * G::E);
#pragma unroll
        for (int q = 0; q < G::NV; ++q) {
            const uint2 a = __ldcg(p + q);
            v[4 * q] = __uint_as_float(a.x << 16);
            v[4 * q + 1] = __uint_as_float(a.x & 0xFFFF0000u);
            v[4 * q + 2] = __uint_as_float(a.y << 16);
            v[4 * q + 3] = __uint_as_float(a.y & 0xFFFF0000u);
        }
    }
}

// MurmurHash3's 32-bit finaliser (Appleby).
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// 64 random bits for the stochastic rounding of the 4 values at columns
// 4 k4 .. 4 k4 + 3 of `row` of table `table_id`, written by the batch that
// starts at sample t0: with the batch's salt s, the SplitMix64 output
// function (Steele, Lea, Flood, OOPSLA 2014) of seed ^ t0 0x9E3779B97F4A7C15
// (the same for every row of the batch, so it is computed once per thread),
// the words w_j = fmix32(lo32(s) + (2 row + table) 0x9E3779B1 + 2 k4 + j),
// j = 0 (low) and 1 (high).
__device__ __forceinline__ uint64_t sr_bits(uint64_t seed, uint32_t table_id, uint64_t row, uint64_t t0, uint32_t k4) {
    uint64_t s = seed ^ (t0 * 0x9E3779B97F4A7C15ull);
    s = (s ^ (s >> 30)) * 0xBF58476D1CE4E5B9ull;
    s = (s ^ (s >> 27)) * 0x94D049BB133111EBull;
    s ^= s >> 31;
    const uint32_t base = (uint32_t)s + (uint32_t)(2 * row + table_id) * 0x9E3779B1u + 2u * k4;
    return ((uint64_t)fmix32(base + 1u) << 32) | fmix32(base);
}

// Store a row part; BF16 rounds stochastically: value i of a 4-value vector
// adds bits [16 i, 16 i + 16) of sr_bits(...) below the BF16 mantissa, then
// truncates (two values per cvt.rs instruction).
template <int D, int DT>
__device__ __forceinline__ void store_row(void* table, int64_t row, int lig, const float (&v)[Geom<D, DT>::E],
                                          uint64_t seed, uint64_t t0, uint32_t table_id) {
    using G = Geom<D, DT>;
    if constexpr (DT == LINE_DTYPE_F32) {
        float4* p = reinterpret_cast<float4*>(reinterpret_cast<float*>(table) + row * D + lig * G::E);
#pragma unroll
        for (int q = 0; q < G::NV; ++q) st_cg(p + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
    } else {
        uint2* p = reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(table) + row * D + lig * G::E);
#pragma unroll
        for (int q = 0; q < G::NV; ++q) {
            const uint32_t k4 = (uint32_t)((lig * G::E + 4 * q) >> 2);
            const uint64_t r = sr_bits(seed, table_id, (uint64_t)row, t0, k4);
            const uint32_t r0 = (uint32_t)r, r1 = (uint32_t)(r >> 32);
            __stcg(p + q, make_uint2(bf16x2_sr(v[4 * q], v[4 * q + 1], r0), bf16x2_sr(v[4 * q + 2], v[4 * q + 3], r1)));
        }
    }
}

template <int L>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = L / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

template <int L>
__device__ __forceinline__ uint32_t group_mask(int grp) {
    return L == 32 ? 0xFFFFFFFFu : (((1u << L) - 1u) << (grp * L));
}

}  // namespace line
