// The library context (line_ctx) and the argument/error helpers shared by the
// C entry points (api.cu, mlp.cu).  Internal: not part of include/line.h.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <string>

#include "line_internal.cuh"

namespace line {

struct Tables {
    void* U = nullptr;
    void* C = nullptr;
    size_t u_cap = 0, c_cap = 0;  // bytes allocated (a later init that fits reuses them)
    int dim = 0;
    int dtype = 0;
    bool ready = false;
};

inline size_t elem_size(int dtype) { return dtype == LINE_DTYPE_F32 ? 4 : 2; }

struct MlpState;  // warm-start network (mlp.cu)
void mlp_destroy(MlpState*);

}  // namespace line

struct line_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    bool sticky = false;
    // graph
    bool has_graph = false;
    int64_t n_nodes = 0, n_arcs = 0;
    int32_t* src = nullptr;
    int32_t* dst = nullptr;
    float* deg = nullptr;  // weighted out-degree of each node (FP64 sum, stored FP32)
    float* w = nullptr;    // arc weights (null: all 1)
    // built on first use for the current graph (the *_ok flags): the first
    // arc of each node (walks, MLP inputs) and the running FP64 weight sums
    // per node (walks); their allocations outlive the graph, like src..deg
    int64_t* row_ptr = nullptr;
    double* cw = nullptr;
    bool row_ptr_ok = false, cw_ok = false;
    size_t row_ptr_cap = 0, cw_cap = 0;
    uint2* edge_tab = nullptr;
    uint2* neg_tab = nullptr;
    // bytes allocated behind src, dst, edge_tab, neg_tab, deg and the weights,
    // and the alias build's scratch: a later graph that fits reuses them
    size_t src_cap = 0, dst_cap = 0, edge_cap = 0, neg_cap = 0, deg_cap = 0, w_cap = 0, x_cap = 0, tmp_cap = 0;
    float* w_buf = nullptr;     // the weights' allocation (w points here for a weighted graph)
    double* alias_x = nullptr;  // alias build scratch
    void* alias_tmp = nullptr;
    // tables by order (index 1 and 2)
    line::Tables tab[3];
    // device status word and small scratch
    uint32_t* status = nullptr;
    uint32_t* flag = nullptr;
    double* dscratch = nullptr;
    line::TrainWorkspace* ws = nullptr;
    // concurrent training of both orders (line_train_orders): the order-1
    // run's workspace and stream, and the events joining it to `stream`
    line::TrainWorkspace* ws2 = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    line::TrainTimes times;
    double total_ms = 0;
    uint64_t total_samples = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    line::MlpState* mlp = nullptr;
};

namespace line {

// Records the message (unless an earlier sticky error is kept) and returns s;
// CUDA and timeout errors make the context sticky.
line_status fail(line_ctx* c, line_status s, const char* fmt, ...);
line_status cuda_fail(line_ctx* c, cudaError_t e, const char* what);
// Entry check: context valid and not sticky, its device current.
line_status enter(line_ctx* c);
// Reads and clears the device status word (synchronises the stream).
line_status check_status(line_ctx* c, const char* what, bool timeout_sticky = true);
// Builds row_ptr if it is missing.
line_status ensure_row_ptr(line_ctx* c);
// Builds the walk sampler tables (row_ptr, cw) if they are missing.
line_status ensure_walk_tables(line_ctx* c);

// An NVTX range over an entry point's host scope (no cost unless a profiler
// is attached; ncu and nsys can filter launches by it).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace line

#define CK(call, what)                                                   \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) return ::line::cuda_fail(c, _e, what);    \
    } while (0)
