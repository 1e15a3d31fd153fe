// Device-wide scans over an index space, used by the alias construction and
// the per-chunk segment build.  Three launches: per-tile reduction, a scan of
// the tile totals in one block, and a per-tile rescan that hands every index
// its exclusive and inclusive prefix to an output functor.  The summation
// order is fixed by the tiling, so integer and FP results are reproducible.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace line {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

// Four counters carried through the alias-pairing scan.
struct Quad {
    uint32_t a, b;
    uint64_t c, d;
    __host__ __device__ Quad operator+(const Quad& o) const { return {a + o.a, b + o.b, c + o.c, d + o.d}; }
};

__device__ __forceinline__ uint32_t shfl_up(uint32_t v, int d) { return __shfl_up_sync(0xFFFFFFFFu, v, d); }
__device__ __forceinline__ uint64_t shfl_up(uint64_t v, int d) {
    return (uint64_t)__shfl_up_sync(0xFFFFFFFFu, (unsigned long long)v, d);
}
__device__ __forceinline__ Quad shfl_up(Quad v, int d) {
    return {shfl_up(v.a, d), shfl_up(v.b, d), shfl_up(v.c, d), shfl_up(v.d, d)};
}
template <typename T>
__device__ __forceinline__ T zero_of() {
    return T{};
}

// Inclusive scan of one value per thread over a block of kScanThreads
// threads; *total receives the block total.  Uses `warp_tot` (>= 32 T) of
// shared memory.
template <typename T>
__device__ T block_inclusive_scan(T v, T* warp_tot, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = shfl_up(v, d);
        if (lane >= d) v = o + v;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (kScanThreads / 32) ? warp_tot[lane] : zero_of<T>();
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T o = shfl_up(w, d);
            if (lane >= d) w = o + w;
        }
        if (lane < (kScanThreads / 32)) warp_tot[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v = warp_tot[warp - 1] + v;
    if (total) *total = warp_tot[kScanThreads / 32 - 1];
    __syncthreads();
    return v;
}

template <typename T, typename Gen>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(int64_t n, Gen gen, T* tile_sums) {
    __shared__ T warp_tot[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T acc = zero_of<T>();
#pragma unroll 4
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        if (i < n) acc = acc + gen(i);
    }
    T total;
    block_inclusive_scan<T>(acc, warp_tot, &total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// One block: exclusive scan of tile_sums in place; the grand total goes to
// *grand (device pointer, may be null).
template <typename T>
__global__ void __launch_bounds__(1024) k_scan_tiles(int64_t ntiles, T* tile_sums, T* grand) {
    __shared__ T part[1024];
    __shared__ T warp_tot[32];
    const int64_t per = (ntiles + 1023) / 1024;
    const int64_t lo = (int64_t)threadIdx.x * per;
    T acc = zero_of<T>();
    for (int64_t i = lo; i < lo + per && i < ntiles; ++i) acc = acc + tile_sums[i];
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        T run = zero_of<T>();
        for (int i = 0; i < 1024; ++i) {
            T v = part[i];
            part[i] = run;
            run = run + v;
        }
        warp_tot[0] = run;
    }
    __syncthreads();
    T run = part[threadIdx.x];
    for (int64_t i = lo; i < lo + per && i < ntiles; ++i) {
        T v = tile_sums[i];
        tile_sums[i] = run;
        run = run + v;
    }
    if (threadIdx.x == 0 && grand) *grand = warp_tot[0];
}

template <typename T, typename Gen, typename Out>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(int64_t n, Gen gen, Out out, const T* tile_offs) {
    __shared__ T warp_tot[32];
    __shared__ T thr_incl[kScanThreads];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T vals[kScanItems];
    T acc = zero_of<T>();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        vals[k] = i < n ? gen(i) : zero_of<T>();
        acc = acc + vals[k];
    }
    thr_incl[threadIdx.x] = block_inclusive_scan<T>(acc, warp_tot, (T*)nullptr);
    __syncthreads();
    // exclusive prefix of this thread's first item
    T excl = tile_offs[blockIdx.x];
    if (threadIdx.x > 0) excl = excl + thr_incl[threadIdx.x - 1];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        const T inc = excl + vals[k];
        if (i < n) out(i, excl, inc);
        excl = inc;
    }
}

inline int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

// tile_buf: scan_tiles(n) + 1 elements of T; the grand total lands in
// tile_buf[scan_tiles(n)].
template <typename T, typename Gen, typename Out>
cudaError_t device_scan(int64_t n, Gen gen, Out out, T* tile_buf, cudaStream_t s) {
    const int64_t nt = scan_tiles(n);
    if (nt == 0) {
        return cudaMemsetAsync(tile_buf, 0, sizeof(T), s);
    }
    k_scan_reduce<T, Gen><<<(unsigned)nt, kScanThreads, 0, s>>>(n, gen, tile_buf);
    k_scan_tiles<T><<<1, 1024, 0, s>>>(nt, tile_buf, tile_buf + nt);
    k_scan_apply<T, Gen, Out><<<(unsigned)nt, kScanThreads, 0, s>>>(n, gen, out, tile_buf);
    return cudaGetLastError();
}

}  // namespace line
