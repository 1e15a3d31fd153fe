// Products of the warm-start MLP with BF16 activations on the tensor cores
// (mlp_fwd.cu).  Forward: C = A W^T for an M x K activation matrix A
// (BF16, row-major) and an N x K FP32 weight matrix W, with
//   hidden layer: A1 = C + b (FP32, optional) and H = GELU(C + b) (BF16);
//   output layer: Y = C (FP32).
// W enters as two BF16 matrices, W_hi = bf16(W) and W_lo = bf16(W - W_hi),
// both multiplied into one FP32 accumulator, so the weights keep about 16
// significant bits in the product (more than TF32's 11), and the BF16
// activations enter exactly.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace line {

// Shapes the kernel takes: N a multiple of 32 up to 256 (two accumulators of
// N columns fill at most the 512 tensor-memory columns), K a multiple of 16,
// and W_hi, W_lo resident in shared memory beside at least two stages of A.
bool fwd_tc_supported(int N, int K);

// BF16 elements of the hi/lo tiles of an N x K weight matrix (2 N K).
inline size_t fwd_w16_elems(int N, int K) { return 2 * (size_t)N * K; }

// W (N x K, row-major FP32) into Wt: W_hi then W_lo, each in the tensor
// core's K-major core-matrix layout (8 rows x 8 values of 16 bytes per core
// matrix, core matrices along K 128 bytes apart, groups of 8 rows 16 K bytes
// apart).
cudaError_t fwd_tile_weights(const float* W, int N, int K, __nv_bfloat16* Wt, cudaStream_t s);

// The product of rows [0, M) of A (row pitch K) with the tiled weights.
// Hidden layer (H != null): bias[N] is added, A1 (nullable) receives the
// sums and H the GELU in BF16.  Output layer (H == null): Y receives the
// sums.  A bounded wait that runs out sets DEV_ERR_TIMEOUT in *status and
// leaves the outputs incomplete.
cudaError_t fwd_tc(int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* Wt, const float* bias, float* A1,
                   __nv_bfloat16* H, float* Y, uint32_t* status, cudaStream_t s);

// dL/da of the hidden layer on the same kernel: dA = (dY W2) * GELU'(A1),
// dY given as its BF16 hi/lo pair (A_hi, A_lo: M x K row-major, K = dim)
// and W2^T tiled by fwd_tile_weights_t (N = hidden); three products per 16
// columns of K (A_hi W_hi, A_hi W_lo, A_lo W_hi).  Writes dA (FP32, M x N)
// and its hi/lo pair (dA_hl: hi, then lo at dA_hl + M N).
bool dact_tc_supported(int N, int K);
cudaError_t dact_tc(int M, int N, int K, const __nv_bfloat16* A_hi, const __nv_bfloat16* A_lo,
                    const __nv_bfloat16* Wt, const float* A1, float* dA, __nv_bfloat16* dA_hl, uint32_t* status,
                    cudaStream_t s);
// The tiles of W^T for W stored K x N row-major (as fwd_tile_weights of the
// transpose).
cudaError_t fwd_tile_weights_t(const float* W, int N, int K, __nv_bfloat16* Wt, cudaStream_t s);

// Weight gradients with BF16 activations: part[z][m][n] = sum over the
// batch rows k of slice z of A[k][m] B[k][n], for A given as its BF16 hi/lo
// pair (A_hi = bf16(A), A_lo = bf16(A - A_hi), each K x M row-major) and B
// BF16 (K x N row-major); the caller sums part[0..wgrad_slices(K)) in slice
// order.  M a multiple of 128, N a multiple of 16 up to 256.  Slices are
// whole multiples of 64 rows, at most kWgradMaxSlices of them.
constexpr int kWgradMaxSlices = 64;
bool wgrad_tc_supported(int M, int N);
int wgrad_slices(int K);
cudaError_t wgrad_tc(int M, int N, int K, const __nv_bfloat16* A_hi, const __nv_bfloat16* A_lo,
                     const __nv_bfloat16* B, float* part, uint32_t* status, cudaStream_t s);

}  // namespace line
