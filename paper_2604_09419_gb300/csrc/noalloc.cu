// Loss evaluation whose scratch lives in a fixed device array, for callers that
// cannot allocate device memory (see line_eval_loss_noalloc in line.h).
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it until the process exits.  In host code its name is only a
// stand-in, not a device address, so the address is looked up once per device
// with cudaGetSymbolAddress (with that device current) and passed to the
// kernels.  line_create does that look-up for its device, so the array is
// loaded and its address known before any entry point runs (under lazy
// module loading the array is created by the first look-up, which may
// allocate).  Every call reuses the same array; nothing in it has to start
// at zero because each call writes every cell it later reads.
#include <mutex>

#include "line_internal.cuh"

namespace line {

namespace {

// m per-sample loss terms, then the block sums of the fixed-order reduction
// of m <= LINE_NOALLOC_MAX_SAMPLES terms.  With at most kSumBlock block sums
// the reduction has one intermediate level, which fits in kSumSlots.
constexpr int64_t kMaxM = LINE_NOALLOC_MAX_SAMPLES;
constexpr int64_t kSumSlots = (kMaxM + kSumBlock - 1) / kSumBlock;
static_assert(kMaxM <= (int64_t)kSumBlock * kSumBlock, "the fixed-order sum would need a second intermediate level");
static __device__ __align__(256) double g_loss_scratch[kMaxM + kSumSlots];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

}  // namespace

cudaError_t noalloc_scratch_address(int device, double** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        double* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_loss_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = p;
    }
    *out = g_addr[device];
    return cudaSuccess;
}

cudaError_t eval_loss_noalloc(int device, const void* U, const void* Ctx, int dtype, int dim, int K,
                              const int32_t* src, const int32_t* dst, const uint2* edge_tab, int64_t n_arcs,
                              const uint2* neg_tab, int64_t n_nodes, uint64_t seed, int64_t m, double* out_dev,
                              cudaStream_t s) {
    if (m < 1 || m > kMaxM) return cudaErrorInvalidValue;
    // the block sums of the one intermediate level must fit in kSumSlots
    const int64_t n_block_sums = (m + kSumBlock - 1) / kSumBlock;
    if (n_block_sums > kSumSlots || n_block_sums > kSumBlock) return cudaErrorInvalidValue;
    double* scratch = nullptr;
    cudaError_t e = noalloc_scratch_address(device, &scratch);
    if (e != cudaSuccess) return e;
    e = eval_loss_terms(U, Ctx, dtype, dim, K, src, dst, edge_tab, n_arcs, neg_tab, n_nodes, seed, m, scratch, s);
    if (e != cudaSuccess) return e;
    return fixed_sum_f64(scratch, m, scratch + kMaxM, out_dev, s);
}

}  // namespace line
