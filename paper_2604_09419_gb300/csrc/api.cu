// C ABI of the LINE library (include/line.h): argument checking, ownership of
// device state, error reporting.  All GPU work is in the other .cu files.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "context.cuh"

using namespace line;

namespace line {

line_status fail(line_ctx* c, line_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        if (c->err.empty() || !c->sticky) c->err = buf;
        if (s == LINE_ERR_CUDA || s == LINE_ERR_TIMEOUT) c->sticky = true;
    }
    return s;
}

line_status cuda_fail(line_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(c, LINE_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(c, LINE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

line_status enter(line_ctx* c) {
    if (!c) return LINE_ERR_ARG;
    if (c->sticky) return LINE_ERR_STATE;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return LINE_OK;
}

line_status check_status(line_ctx* c, const char* what, bool timeout_sticky) {
    uint32_t st = 0;
    CK(cudaMemcpyAsync(&st, c->status, sizeof st, cudaMemcpyDeviceToHost, c->stream), "status read");
    CK(cudaStreamSynchronize(c->stream), what);
    if (st) CK(cudaMemsetAsync(c->status, 0, sizeof(uint32_t), c->stream), "status reset");
    if (st & DEV_ERR_GRAPH) return fail(c, LINE_ERR_VALIDATE, "%s: graph validation failed", what);
    if (st & DEV_ERR_ALIAS) return fail(c, LINE_ERR_VALIDATE, "%s: alias construction invariant failed", what);
    if (st & DEV_ERR_TIMEOUT) {
        if (timeout_sticky) return fail(c, LINE_ERR_TIMEOUT, "%s: device wait exceeded the spin limit", what);
        return LINE_ERR_TIMEOUT;
    }
    if (st & DEV_ERR_INDEX) return fail(c, LINE_ERR_ARG, "%s: index out of range", what);
    if (st & DEV_ERR_VALUE) return fail(c, LINE_ERR_VALIDATE, "%s: non-finite value", what);
    return LINE_OK;
}

// *p holds at least `bytes` (a larger earlier allocation is kept).
template <typename T>
cudaError_t grow(T** p, size_t* cap, size_t bytes) {
    if (*p && *cap >= bytes) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e == cudaSuccess) *cap = bytes;
    return e;
}

line_status ensure_row_ptr(line_ctx* c) {
    if (c->row_ptr_ok) return LINE_OK;
    cudaError_t e = grow(&c->row_ptr, &c->row_ptr_cap, sizeof(int64_t) * (size_t)(c->n_nodes + 1));
    if (e == cudaSuccess) e = row_offsets(c->n_nodes, c->n_arcs, c->src, c->row_ptr, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "row offsets");
    c->row_ptr_ok = true;
    return LINE_OK;
}

line_status ensure_walk_tables(line_ctx* c) {
    if (c->cw_ok) return LINE_OK;
    line_status st = ensure_row_ptr(c);
    if (st) return st;
    cudaError_t e = grow(&c->cw, &c->cw_cap, sizeof(double) * (size_t)std::max<int64_t>(1, c->n_arcs));
    if (e == cudaSuccess) e = walk_cumw(c->n_nodes, c->row_ptr, c->w, c->cw, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "walk sampler tables");
    c->cw_ok = true;
    return LINE_OK;
}


}  // namespace line

namespace {

void free_tables(Tables& t) {
    if (t.U) cudaFree(t.U);
    if (t.C) cudaFree(t.C);
    t = Tables{};
}

// The graph is gone: its row offsets and walk tables are out of date (they
// are built again for the next graph on first use); the graph, alias and
// walk buffers stay allocated for the next build (release_graph frees them).
void free_graph(line_ctx* c, bool keep_tables = false) {
    c->row_ptr_ok = c->cw_ok = false;
    c->w = nullptr;
    c->has_graph = false;
    if (keep_tables) return;
    mlp_destroy(c->mlp);
    c->mlp = nullptr;
    for (auto& t : c->tab) free_tables(t);
}

void release_graph(line_ctx* c) {
    free_graph(c);
    for (void* p : {(void*)c->src, (void*)c->dst, (void*)c->deg, (void*)c->edge_tab, (void*)c->neg_tab, (void*)c->w_buf,
                    (void*)c->alias_x, c->alias_tmp, (void*)c->row_ptr, (void*)c->cw})
        if (p) cudaFree(p);
    c->row_ptr = nullptr;
    c->cw = nullptr;
    c->row_ptr_cap = c->cw_cap = 0;
    c->src = c->dst = nullptr;
    c->deg = nullptr;
    c->edge_tab = c->neg_tab = nullptr;
    c->w_buf = nullptr;
    c->alias_x = nullptr;
    c->alias_tmp = nullptr;
    c->src_cap = c->dst_cap = c->edge_cap = c->neg_cap = c->deg_cap = c->w_cap = c->x_cap = c->tmp_cap = 0;
}

bool dim_ok(int dim) { return dim == 16 || dim == 32 || dim == 64 || dim == 128 || dim == 256; }

}  // namespace

extern "C" {

void line_train_opts_default(line_train_opts* o) {
    if (!o) return;
    o->batch = 4096;
    o->lambda = 0.0;
    o->alpha_neg = 1.0;
    o->sample_offset = 0;
    o->mode = LINE_MODE_BATCHED;
    o->spin_limit = 0;
    o->chunk_batches = 0;
    o->warps_per_block = 0;
    o->timing = 0;
    o->graph = 1;
    o->walk_length = 0;
    o->window = 0;
    o->walk_reuse = 1;
    o->hogwild_workers = 0;
}

const char* line_status_string(line_status s) {
    switch (s) {
        case LINE_OK: return "ok";
        case LINE_ERR_ARG: return "invalid argument";
        case LINE_ERR_OOM: return "out of device memory";
        case LINE_ERR_CUDA: return "CUDA error";
        case LINE_ERR_TIMEOUT: return "device wait timed out";
        case LINE_ERR_STATE: return "invalid state";
        case LINE_ERR_VALIDATE: return "validation failed";
    }
    return "unknown status";
}

line_status line_create(line_ctx** out, int device, void* cuda_stream) {
    if (!out) return LINE_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return LINE_ERR_ARG;
    }
    line_ctx* c = new line_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&c->status, 256) != cudaSuccess ||
        cudaMemset(c->status, 0, 256) != cudaSuccess || cudaMalloc(&c->dscratch, 64) != cudaSuccess ||
        cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
        cudaGetLastError();
        line_destroy(c);
        return LINE_ERR_CUDA;
    }
    c->flag = c->status + 32;  // never set: target of line_debug_wait_timeout
    // load the fixed array of line_eval_loss_noalloc on this device now, so
    // that its callers never trigger a module load or allocation later
    double* noalloc_scratch = nullptr;
    if (noalloc_scratch_address(device, &noalloc_scratch) != cudaSuccess) {
        cudaGetLastError();
        line_destroy(c);
        return LINE_ERR_CUDA;
    }
    c->ws = workspace_create();
    *out = c;
    return LINE_OK;
}

void line_destroy(line_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    release_graph(c);
    workspace_destroy(c->ws);
    workspace_destroy(c->ws2);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->status) cudaFree(c->status);
    if (c->dscratch) cudaFree(c->dscratch);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    cudaGetLastError();
    delete c;
}

const char* line_last_error(const line_ctx* c) { return c ? c->err.c_str() : "null context"; }

line_status line_build_alias(line_ctx* c, const line_graph_desc* g) {
    NvtxRange nvtx("line_build_alias");
    line_status st = enter(c);
    if (st) return st;
    if (!g || !g->src || !g->dst) return fail(c, LINE_ERR_ARG, "line_build_alias: null graph arrays");
    if (g->n_nodes < 1 || g->n_nodes >= (1ll << 30)) return fail(c, LINE_ERR_ARG, "line_build_alias: n_nodes out of range");
    if (g->n_arcs < 1 || g->n_arcs >= (1ll << 32) - 1) return fail(c, LINE_ERR_ARG, "line_build_alias: n_arcs out of range");
    // tables (and the MLP) survive a graph of the same node count
    const bool keep = c->has_graph && c->n_nodes == g->n_nodes;
    free_graph(c, keep);
    const int64_t n = g->n_nodes, m = g->n_arcs;
    cudaStream_t s = c->stream;
    // the buffers of an earlier graph are reused when large enough; the
    // work queued on the stream before this call may still read them, and
    // the stream orders it before the copies below
    CK(grow(&c->src, &c->src_cap, sizeof(int32_t) * m), "graph allocation");
    CK(grow(&c->dst, &c->dst_cap, sizeof(int32_t) * m), "graph allocation");
    CK(grow(&c->edge_tab, &c->edge_cap, sizeof(uint2) * m), "alias allocation");
    CK(grow(&c->neg_tab, &c->neg_cap, sizeof(uint2) * n), "alias allocation");
    CK(grow(&c->deg, &c->deg_cap, sizeof(float) * n), "degree allocation");
    CK(cudaMemcpyAsync(c->src, g->src, sizeof(int32_t) * m, cudaMemcpyDefault, s), "graph copy");
    CK(cudaMemcpyAsync(c->dst, g->dst, sizeof(int32_t) * m, cudaMemcpyDefault, s), "graph copy");
    float* w = nullptr;
    line_status result = LINE_OK;
    do {
        cudaError_t e;
        if (g->w) {
            if ((e = grow(&c->w_buf, &c->w_cap, sizeof(float) * m)) != cudaSuccess) { result = cuda_fail(c, e, "weights"); break; }
            w = c->w_buf;
            if ((e = cudaMemcpyAsync(w, g->w, sizeof(float) * m, cudaMemcpyDefault, s)) != cudaSuccess) {
                result = cuda_fail(c, e, "weights copy");
                break;
            }
        }
        if ((e = validate_graph(n, m, c->src, c->dst, w, c->status, s)) != cudaSuccess) { result = cuda_fail(c, e, "validate"); break; }
        if ((result = check_status(c, "line_build_alias"))) break;
        const int64_t big = n > m ? n : m;
        if ((e = grow(&c->alias_x, &c->x_cap, sizeof(double) * big)) != cudaSuccess) { result = cuda_fail(c, e, "alias scratch"); break; }
        if ((e = grow(&c->alias_tmp, &c->tmp_cap, alias_build_tmp_bytes(big))) != cudaSuccess) { result = cuda_fail(c, e, "alias scratch"); break; }
        double* x = c->alias_x;
        void* tmp = c->alias_tmp;
        // edge table: arc weights (Algorithm 3)
        if ((e = edge_weights(m, w, x, s)) != cudaSuccess) { result = cuda_fail(c, e, "edge weights"); break; }
        if ((e = alias_build(x, m, c->edge_tab, tmp, c->status, s)) != cudaSuccess) { result = cuda_fail(c, e, "edge alias"); break; }
        if ((result = check_status(c, "line_build_alias (edges)"))) break;
        // negative table: d(v)^0.75 (Eq. 1), each node's arcs found by the
        // row offsets (kept for the walk sampler and the MLP inputs)
        if ((e = grow(&c->row_ptr, &c->row_ptr_cap, sizeof(int64_t) * (size_t)(n + 1))) != cudaSuccess) { result = cuda_fail(c, e, "row offsets"); break; }
        if ((e = row_offsets(n, m, c->src, c->row_ptr, s)) != cudaSuccess) { result = cuda_fail(c, e, "row offsets"); break; }
        if ((e = neg_weights(n, m, c->row_ptr, w, x, c->deg, c->flag + 1, s)) != cudaSuccess) { result = cuda_fail(c, e, "degree weights"); break; }
        if ((e = alias_build(x, n, c->neg_tab, tmp, c->status, s)) != cudaSuccess) { result = cuda_fail(c, e, "negative alias"); break; }
        if ((result = check_status(c, "line_build_alias (negatives)"))) break;
    } while (false);
    c->w = w;  // kept for the walk sampler's tables (null: unit weights)
    if (result != LINE_OK) {
        cudaStreamSynchronize(s);
        free_graph(c);
        return result;
    }
    c->n_nodes = n;
    c->n_arcs = m;
    c->has_graph = true;
    c->row_ptr_ok = true;
    return LINE_OK;
}

line_status line_get_graph_info(line_ctx* c, int64_t* n_nodes, int64_t* n_arcs) {
    line_status st = enter(c);
    if (st) return st;
    if (!c->has_graph) return fail(c, LINE_ERR_STATE, "no graph");
    if (n_nodes) *n_nodes = c->n_nodes;
    if (n_arcs) *n_arcs = c->n_arcs;
    return LINE_OK;
}

line_status line_get_alias(line_ctx* c, int table, uint32_t* thr, uint32_t* alias) {
    line_status st = enter(c);
    if (st) return st;
    if (!c->has_graph) return fail(c, LINE_ERR_STATE, "line_get_alias: no graph");
    if ((table != LINE_TABLE_EDGE && table != LINE_TABLE_NEG) || !thr || !alias)
        return fail(c, LINE_ERR_ARG, "line_get_alias: bad arguments");
    const int64_t n = table == LINE_TABLE_EDGE ? c->n_arcs : c->n_nodes;
    const uint2* tab = table == LINE_TABLE_EDGE ? c->edge_tab : c->neg_tab;
    uint32_t* buf = nullptr;
    CK(cudaMalloc(&buf, sizeof(uint32_t) * 2 * n), "alias export scratch");
    cudaError_t e = export_alias(tab, n, buf, buf + n, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(thr, buf, sizeof(uint32_t) * n, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(alias, buf + n, sizeof(uint32_t) * n, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(c, e, "line_get_alias");
    return LINE_OK;
}

line_status line_sample_debug(line_ctx* c, int K, uint64_t seed, uint32_t domain, uint64_t t0, int64_t count,
                              int32_t* out) {
    NvtxRange nvtx("line_sample_debug");
    line_status st = enter(c);
    if (st) return st;
    if (!c->has_graph) return fail(c, LINE_ERR_STATE, "line_sample_debug: no graph");
    if (K < 0 || K > kMaxK || count < 0 || (!out && count > 0)) return fail(c, LINE_ERR_ARG, "line_sample_debug: bad arguments");
    if (count == 0) return LINE_OK;
    int32_t* buf = nullptr;
    const size_t bytes = sizeof(int32_t) * (size_t)count * (K + 2);
    cudaPointerAttributes attr;
    bool dev_out = cudaPointerGetAttributes(&attr, out) == cudaSuccess && attr.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    if (!dev_out) CK(cudaMalloc(&buf, bytes), "sample scratch");
    cudaError_t e = sample_records(c->src, c->dst, c->edge_tab, c->n_arcs, c->neg_tab, c->n_nodes, seed, domain, t0,
                                   count, K, dev_out ? out : buf, c->stream);
    if (e == cudaSuccess && !dev_out) e = cudaMemcpyAsync(out, buf, bytes, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (buf) cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(c, e, "line_sample_debug");
    return LINE_OK;
}

line_status line_sample_walk_debug(line_ctx* c, int K, uint64_t seed, int walk_length, int window, int reuse,
                                   uint64_t t0, int64_t count, int32_t* out) {
    NvtxRange nvtx("line_sample_walk_debug");
    line_status st = enter(c);
    if (st) return st;
    if (!c->has_graph) return fail(c, LINE_ERR_STATE, "line_sample_walk_debug: no graph");
    if (K < 0 || K > kMaxK || count < 0 || (!out && count > 0))
        return fail(c, LINE_ERR_ARG, "line_sample_walk_debug: bad arguments");
    if (walk_length < 1 || walk_length > kMaxWalkLen || window < 1 || window > walk_length)
        return fail(c, LINE_ERR_ARG, "line_sample_walk_debug: need 1 <= window <= walk_length <= %d", kMaxWalkLen);
    if (reuse < 1 || reuse > kMaxWalkReuse)
        return fail(c, LINE_ERR_ARG, "line_sample_walk_debug: need 1 <= reuse <= %d", kMaxWalkReuse);
    if (count == 0) return LINE_OK;
    if ((st = ensure_walk_tables(c))) return st;
    int32_t* buf = nullptr;
    const size_t bytes = sizeof(int32_t) * (size_t)count * (K + 2);
    cudaPointerAttributes attr;
    bool dev_out = cudaPointerGetAttributes(&attr, out) == cudaSuccess && attr.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    if (!dev_out) CK(cudaMalloc(&buf, bytes), "sample scratch");
    int32_t* rec = dev_out ? out : buf;
    // negatives: the edge sampler's draws (domain 0, calls 1..K); its slots 0
    // and 1 are then overwritten by the walk pairs
    cudaError_t e = sample_records(c->src, c->dst, c->edge_tab, c->n_arcs, c->neg_tab, c->n_nodes, seed, 0u, t0,
                                   count, K, rec, c->stream);
    if (e == cudaSuccess) {
        WalkParams wp{};
        wp.src = c->src;
        wp.dst = c->dst;
        wp.edge_tab = c->edge_tab;
        wp.n_arcs = c->n_arcs;
        wp.row_ptr = c->row_ptr;
        wp.cw = c->cw;
        wp.seed = seed;
        wp.t0 = t0;
        wp.count = count;
        wp.L = walk_length;
        wp.W = window;
        wp.P = (uint64_t)walk_length * window - (uint64_t)window * (window - 1) / 2;
        wp.reuse = (uint32_t)reuse;
        wp.R = (uint64_t)(K + 2);
        wp.rec = rec;
        e = walk_pairs(wp, c->stream);
    }
    if (e == cudaSuccess && !dev_out) e = cudaMemcpyAsync(out, buf, bytes, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (buf) cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(c, e, "line_sample_walk_debug");
    return LINE_OK;
}

line_status line_init_embeddings(line_ctx* c, int order, int dim, int dtype, uint64_t seed) {
    NvtxRange nvtx("line_init_embeddings");
    line_status st = enter(c);
    if (st) return st;
    if (!c->has_graph) return fail(c, LINE_ERR_STATE, "line_init_embeddings: no graph");
    if ((order != 1 && order != 2) || !dim_ok(dim) || (dtype != LINE_DTYPE_F32 && dtype != LINE_DTYPE_BF16))
        return fail(c, LINE_ERR_ARG, "line_init_embeddings: bad order/dim/dtype");
    Tables& t = c->tab[order];
    t.ready = false;
    // the tables' earlier allocations are reused when they are large enough
    const size_t bytes = (size_t)c->n_nodes * dim * elem_size(dtype);
    cudaError_t e = grow(&t.U, &t.u_cap, bytes);
    if (e == cudaSuccess) e = init_table(t.U, dtype, c->n_nodes, dim, seed, c->stream);
    if (e == cudaSuccess && order == 2) e = grow(&t.C, &t.c_cap, bytes);
    if (e == cudaSuccess && order == 2) e = cudaMemsetAsync(t.C, 0, bytes, c->stream);
    if (e != cudaSuccess) {
        free_tables(t);  // nothing of a failed call is kept
        return cuda_fail(c, e, "line_init_embeddings: table allocation");
    }
    t.dim = dim;
    t.dtype = dtype;
    t.ready = true;
    return LINE_OK;
}

}  // extern "C"

namespace {

// Checks the arguments of a training call and fills the kernel arguments.
line_status make_train_args(line_ctx* c, const char* what, int order, int dim, int K, const line_lr* lr,
                            uint64_t n_samples, uint64_t seed, const line_train_opts* opts, TrainArgs* out) {
    if (!c->has_graph) return fail(c, LINE_ERR_STATE, "%s: no graph", what);
    if (order != 1 && order != 2) return fail(c, LINE_ERR_ARG, "%s: order must be 1 or 2", what);
    Tables& t = c->tab[order];
    if (!t.ready || t.dim != dim)
        return fail(c, LINE_ERR_STATE, "%s: tables of order %d and dim %d not initialised", what, order, dim);
    if (K < 0 || K > kMaxK) return fail(c, LINE_ERR_ARG, "%s: K out of range", what);
    if (!lr || !(lr->lr0 >= 0.0) || (lr->schedule != 0 && lr->schedule != 1) || !(lr->floor_frac >= 0.0))
        return fail(c, LINE_ERR_ARG, "%s: bad learning rate", what);
    line_train_opts o;
    line_train_opts_default(&o);
    if (opts) o = *opts;
    if (o.batch < 1 || o.batch > (1 << 20)) return fail(c, LINE_ERR_ARG, "%s: batch out of range", what);
    if (!(o.lambda >= 0.0) || !(o.alpha_neg >= 0.0)) return fail(c, LINE_ERR_ARG, "%s: bad lambda/alpha_neg", what);
    if (o.mode != LINE_MODE_BATCHED && o.mode != LINE_MODE_PERSISTENT && o.mode != LINE_MODE_HOGWILD)
        return fail(c, LINE_ERR_ARG, "%s: bad mode", what);
    if (o.hogwild_workers < 0) return fail(c, LINE_ERR_ARG, "%s: hogwild_workers must be >= 0", what);
    if (o.warps_per_block < 0 || o.warps_per_block > 32) return fail(c, LINE_ERR_ARG, "%s: bad warps_per_block", what);
    if (o.sample_offset + n_samples < o.sample_offset) return fail(c, LINE_ERR_ARG, "%s: sample range overflows", what);
    if (o.walk_length < 0 || o.walk_length > kMaxWalkLen ||
        (o.walk_length > 0 && (o.window < 1 || o.window > o.walk_length)))
        return fail(c, LINE_ERR_ARG, "%s: need 1 <= window <= walk_length <= %d", what, kMaxWalkLen);
    if (o.walk_reuse < 0 || o.walk_reuse > kMaxWalkReuse)
        return fail(c, LINE_ERR_ARG, "%s: need 0 <= walk_reuse <= %d", what, kMaxWalkReuse);
    if (o.walk_length > 0) {
        line_status ws = ensure_walk_tables(c);
        if (ws) return ws;
    }
    TrainArgs a{};
    a.order = order;
    a.dim = dim;
    a.K = K;
    a.dtype = t.dtype;
    a.n_nodes = c->n_nodes;
    a.n_arcs = c->n_arcs;
    a.src = c->src;
    a.dst = c->dst;
    a.edge_tab = c->edge_tab;
    a.neg_tab = c->neg_tab;
    a.U = t.U;
    a.C = t.C;
    a.seed = seed;
    a.t_begin = o.sample_offset;
    a.t_end = o.sample_offset + n_samples;
    a.batch = o.batch;
    a.lr0 = lr->lr0;
    a.lr_floor = lr->floor_frac;
    a.lr_schedule = lr->schedule;
    a.lr_total = lr->total ? lr->total : o.sample_offset + n_samples;
    a.lambda = o.lambda;
    a.alpha_neg = o.alpha_neg;
    a.mode = o.mode;
    a.spin_limit = o.spin_limit > 0 ? o.spin_limit : (int64_t)1 << 22;  // ~1 s of polling
    a.chunk_batches = o.chunk_batches;
    a.warps_per_block = o.warps_per_block;
    a.timing = o.timing;
    a.hogwild_workers = o.hogwild_workers;
    a.walk_len = o.walk_length;
    a.window = o.walk_length > 0 ? o.window : 0;
    a.walk_reuse = o.walk_reuse > 0 ? o.walk_reuse : 1;
    a.row_ptr = o.walk_length > 0 ? c->row_ptr : nullptr;
    a.cw = o.walk_length > 0 ? c->cw : nullptr;
    a.graph = o.graph;
    *out = a;
    return LINE_OK;
}

line_status train_fail(line_ctx* c, cudaError_t e, const std::string& err, const char* what) {
    if (!err.empty()) return fail(c, e == cudaErrorMemoryAllocation ? LINE_ERR_OOM : LINE_ERR_ARG, "%s: %s", what, err.c_str());
    return cuda_fail(c, e, what);
}

}  // namespace

extern "C" {

line_status line_train_steps(line_ctx* c, int order, int dim, int K, const line_lr* lr, uint64_t n_samples,
                             uint64_t seed, const line_train_opts* opts) {
    NvtxRange nvtx("line_train_steps");
    line_status st = enter(c);
    if (st) return st;
    TrainArgs a{};
    if ((st = make_train_args(c, "line_train_steps", order, dim, K, lr, n_samples, seed, opts, &a))) return st;
    if (n_samples == 0) return LINE_OK;
    std::string err;
    if (a.timing) CK(cudaEventRecord(c->ev0, c->stream), "event");
    cudaError_t e = train_run(a, c->ws, c->status, &c->times, c->stream, &err);
    if (e != cudaSuccess) return train_fail(c, e, err, "line_train_steps");
    if (a.timing) CK(cudaEventRecord(c->ev1, c->stream), "event");
    st = check_status(c, "line_train_steps");
    if (st) return st;
    if (a.timing) {
        float ms = 0;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        c->total_ms += ms;
        c->total_samples += n_samples;
    }
    return LINE_OK;
}

line_status line_train_orders(line_ctx* c, int dim, int K, const line_lr* lr, uint64_t n_samples, uint64_t seed,
                              const line_train_opts* opts) {
    NvtxRange nvtx("line_train_orders");
    line_status st = enter(c);
    if (st) return st;
    TrainArgs a1{}, a2{};
    if ((st = make_train_args(c, "line_train_orders", 1, dim, K, lr, n_samples, seed, opts, &a1))) return st;
    if ((st = make_train_args(c, "line_train_orders", 2, dim, K, lr, n_samples, seed, opts, &a2))) return st;
    if (n_samples == 0) return LINE_OK;
    // per-chunk timing reads events on the host between chunks, which would
    // serialise the two streams: the call is timed as a whole instead
    const bool timing = a1.timing != 0;
    a1.timing = a2.timing = 0;
    a1.concurrent = a2.concurrent = true;
    if (!c->ws2) c->ws2 = workspace_create();
    if (!c->side) CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "line_train_orders: stream");
    if (!c->ev_fork) CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "line_train_orders: event");
    if (!c->ev_join) CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "line_train_orders: event");
    if (timing) CK(cudaEventRecord(c->ev0, c->stream), "event");
    // order 1 on the side stream, after the caller's earlier work
    CK(cudaEventRecord(c->ev_fork, c->stream), "line_train_orders: fork");
    CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0), "line_train_orders: fork");
    std::string err;
    // Both orders in alternate slices of about 2^24 samples (whole pre-pass
    // chunks): order 1's slice on the side stream, then order 2's.  The
    // launch queues then always hold work of both orders.  Enqueuing one
    // order's whole run first would, once a long run fills the queues, hold
    // the host inside order 1 and train the orders one after the other.
    // Splitting at whole batches leaves the tables bitwise unchanged.
    const uint64_t chunk =
        (uint64_t)(a1.chunk_batches > 0 ? a1.chunk_batches : std::max<int64_t>(1, ((int64_t)1 << 18) / a1.batch)) *
        (uint64_t)a1.batch;
    const uint64_t slice = std::max<uint64_t>(chunk, ((uint64_t)1 << 24) / chunk * chunk);
    cudaError_t e = cudaSuccess;
    for (uint64_t t0 = a1.t_begin; t0 < a1.t_end && e == cudaSuccess; t0 += slice) {
        TrainArgs s1 = a1, s2 = a2;
        s1.t_begin = s2.t_begin = t0;
        s1.t_end = s2.t_end = std::min<uint64_t>(a1.t_end, t0 + slice);
        e = train_run(s1, c->ws2, c->status, &c->times, c->side, &err);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(c->side);
            return train_fail(c, e, err, "line_train_orders");
        }
        e = train_run(s2, c->ws, c->status, &c->times, c->stream, &err);
    }
    // the caller's stream continues after both
    cudaError_t ej = cudaEventRecord(c->ev_join, c->side);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(c->stream, c->ev_join, 0);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(c->side);
        return train_fail(c, e, err, "line_train_orders");
    }
    CK(ej, "line_train_orders: join");
    if (timing) CK(cudaEventRecord(c->ev1, c->stream), "event");
    st = check_status(c, "line_train_orders");
    if (st) return st;
    if (timing) {
        float ms = 0;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        c->total_ms += ms;
        c->total_samples += 2 * n_samples;
    }
    return LINE_OK;
}

line_status line_get_embeddings(line_ctx* c, int order, int which, void* dst, int dst_dtype) {
    NvtxRange nvtx("line_get_embeddings");
    line_status st = enter(c);
    if (st) return st;
    if (order != 1 && order != 2) return fail(c, LINE_ERR_ARG, "line_get_embeddings: bad order");
    Tables& t = c->tab[order];
    if (!t.ready) return fail(c, LINE_ERR_STATE, "line_get_embeddings: no tables of order %d", order);
    if (!dst || (which != LINE_WHICH_U && which != LINE_WHICH_C) || (which == LINE_WHICH_C && order != 2))
        return fail(c, LINE_ERR_ARG, "line_get_embeddings: bad arguments");
    if (dst_dtype != LINE_DTYPE_F32 && !(dst_dtype == LINE_DTYPE_BF16 && t.dtype == LINE_DTYPE_BF16))
        return fail(c, LINE_ERR_ARG, "line_get_embeddings: unsupported dtype conversion");
    const void* srcp = which == LINE_WHICH_U ? t.U : t.C;
    const size_t elems = (size_t)c->n_nodes * t.dim;
    if (dst_dtype == t.dtype) {
        CK(cudaMemcpyAsync(dst, srcp, elems * elem_size(t.dtype), cudaMemcpyDefault, c->stream), "embedding copy");
    } else {
        void* buf = nullptr;
        CK(cudaMalloc(&buf, elems * 4), "conversion scratch");
        cudaError_t e = convert_rows(srcp, t.dtype, buf, LINE_DTYPE_F32, nullptr, c->n_nodes, t.dim, c->n_nodes,
                                     c->status, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, buf, elems * 4, cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(buf);
        if (e != cudaSuccess) return cuda_fail(c, e, "line_get_embeddings");
    }
    CK(cudaStreamSynchronize(c->stream), "line_get_embeddings");
    return LINE_OK;
}

line_status line_set_embeddings(line_ctx* c, int order, int which, const void* src, int src_dtype,
                                const int32_t* rows, int64_t n_rows) {
    NvtxRange nvtx("line_set_embeddings");
    line_status st = enter(c);
    if (st) return st;
    if (order != 1 && order != 2) return fail(c, LINE_ERR_ARG, "line_set_embeddings: bad order");
    Tables& t = c->tab[order];
    if (!t.ready) return fail(c, LINE_ERR_STATE, "line_set_embeddings: no tables of order %d", order);
    if ((which != LINE_WHICH_U && which != LINE_WHICH_C) || (which == LINE_WHICH_C && order != 2) ||
        (src_dtype != LINE_DTYPE_F32 && src_dtype != LINE_DTYPE_BF16) || n_rows < 0 || (n_rows > 0 && !src) ||
        (!rows && n_rows > c->n_nodes))
        return fail(c, LINE_ERR_ARG, "line_set_embeddings: bad arguments");
    if (n_rows == 0) return LINE_OK;
    void* dstp = which == LINE_WHICH_U ? t.U : t.C;
    const size_t in_bytes = (size_t)n_rows * t.dim * elem_size(src_dtype);
    void* sbuf = nullptr;
    int32_t* rbuf = nullptr;
    cudaError_t e = cudaMalloc(&sbuf, in_bytes);
    if (e == cudaSuccess && rows) e = cudaMalloc(&rbuf, sizeof(int32_t) * n_rows);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sbuf, src, in_bytes, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && rows) e = cudaMemcpyAsync(rbuf, rows, sizeof(int32_t) * n_rows, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess)
        e = convert_rows(sbuf, src_dtype, dstp, t.dtype, rbuf, n_rows, t.dim, c->n_nodes, c->status, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (sbuf) cudaFree(sbuf);
    if (rbuf) cudaFree(rbuf);
    if (e != cudaSuccess) return cuda_fail(c, e, "line_set_embeddings");
    return check_status(c, "line_set_embeddings");
}

line_status line_eval_loss(line_ctx* c, int order, int K, uint64_t seed, int64_t m, double* out_host) {
    NvtxRange nvtx("line_eval_loss");
    line_status st = enter(c);
    if (st) return st;
    if (!c->has_graph) return fail(c, LINE_ERR_STATE, "line_eval_loss: no graph");
    if (order != 1 && order != 2) return fail(c, LINE_ERR_ARG, "line_eval_loss: bad order");
    Tables& t = c->tab[order];
    if (!t.ready) return fail(c, LINE_ERR_STATE, "line_eval_loss: no tables of order %d", order);
    if (K < 0 || K > kMaxK || m < 0 || !out_host) return fail(c, LINE_ERR_ARG, "line_eval_loss: bad arguments");
    if (m == 0) {
        *out_host = 0.0;
        return LINE_OK;
    }
    double* terms = nullptr;
    void* tmp = nullptr;
    cudaError_t e = cudaMalloc(&terms, sizeof(double) * m);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, fixed_sum_tmp_bytes(m));
    if (e == cudaSuccess)
        e = eval_loss_terms(t.U, order == 2 ? t.C : t.U, t.dtype, t.dim, K, c->src, c->dst, c->edge_tab, c->n_arcs,
                            c->neg_tab, c->n_nodes, seed, m, terms, c->stream);
    if (e == cudaSuccess) e = fixed_sum_f64(terms, m, (double*)tmp, c->dscratch, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, c->dscratch, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (terms) cudaFree(terms);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "line_eval_loss");
    return LINE_OK;
}

line_status line_eval_auc(line_ctx* c, int orders, int score, const int32_t* pos_src, const int32_t* pos_dst, int64_t n_pos,
                          const int32_t* neg_src, const int32_t* neg_dst, int64_t n_neg, float* scores_out,
                          uint64_t* counts_out, double* auc_out) {
    NvtxRange nvtx("line_eval_auc");
    line_status st = enter(c);
    if (st) return st;
    if (!c->has_graph) return fail(c, LINE_ERR_STATE, "line_eval_auc: no graph");
    if (orders < 1 || orders > 3 || (score != LINE_SCORE_DOT && score != LINE_SCORE_COSINE) || n_pos < 1 || n_neg < 1 || n_pos + n_neg >= (1ll << 31) || !pos_src || !pos_dst ||
        !neg_src || !neg_dst || !auc_out)
        return fail(c, LINE_ERR_ARG, "line_eval_auc: bad arguments");
    ScoreTables t{};
    for (int o = 1; o <= 2; ++o) {
        if (!(orders & o)) continue;
        if (!c->tab[o].ready) return fail(c, LINE_ERR_STATE, "line_eval_auc: no tables of order %d", o);
        t.U[t.n] = c->tab[o].U;
        t.dim[t.n] = c->tab[o].dim;
        t.dtype[t.n] = c->tab[o].dtype;
        ++t.n;
    }
    const int64_t n = n_pos + n_neg;
    int32_t* pairs = nullptr;
    float* scores = nullptr;
    void* tmp = nullptr;
    unsigned long long counts[2] = {0, 0};
    cudaStream_t s = c->stream;
    cudaError_t e = cudaMalloc(&pairs, sizeof(int32_t) * 2 * n);
    if (e == cudaSuccess) e = cudaMalloc(&scores, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, auc_tmp_bytes(n_pos, n_neg));
    int32_t* src = pairs;
    int32_t* dst = pairs + n;
    if (e == cudaSuccess) e = cudaMemcpyAsync(src, pos_src, sizeof(int32_t) * n_pos, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(src + n_pos, neg_src, sizeof(int32_t) * n_neg, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, pos_dst, sizeof(int32_t) * n_pos, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst + n_pos, neg_dst, sizeof(int32_t) * n_neg, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = eval_auc(t, score, src, dst, n_pos, n_neg, c->n_nodes, scores, tmp, c->status, s);
    if (e == cudaSuccess && scores_out)
        e = cudaMemcpyAsync(scores_out, scores, sizeof(float) * n, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, tmp, sizeof counts, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (pairs) cudaFree(pairs);
    if (scores) cudaFree(scores);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "line_eval_auc");
    if ((st = check_status(c, "line_eval_auc"))) return st;
    if (counts_out) {
        counts_out[0] = counts[0];
        counts_out[1] = counts[1];
    }
    *auc_out = (double)(2 * counts[0] + counts[1]) / (2.0 * (double)n_pos * (double)n_neg);
    return LINE_OK;
}

line_status line_eval_loss_noalloc(line_ctx* c, int order, int K, uint64_t seed, int64_t m, double* out_host) {
    NvtxRange nvtx("line_eval_loss_noalloc");
    line_status st = enter(c);
    if (st) return st;
    if (!c->has_graph) return fail(c, LINE_ERR_STATE, "line_eval_loss_noalloc: no graph");
    if (order != 1 && order != 2) return fail(c, LINE_ERR_ARG, "line_eval_loss_noalloc: bad order");
    Tables& t = c->tab[order];
    if (!t.ready) return fail(c, LINE_ERR_STATE, "line_eval_loss_noalloc: no tables of order %d", order);
    if (K < 0 || K > kMaxK || !out_host) return fail(c, LINE_ERR_ARG, "line_eval_loss_noalloc: bad arguments");
    if (m < 1 || m > LINE_NOALLOC_MAX_SAMPLES)
        return fail(c, LINE_ERR_ARG, "line_eval_loss_noalloc: m = %lld outside 1..%d (the fixed scratch size)",
                    (long long)m, LINE_NOALLOC_MAX_SAMPLES);
    CK(eval_loss_noalloc(c->device, t.U, order == 2 ? t.C : t.U, t.dtype, t.dim, K, c->src, c->dst, c->edge_tab,
                         c->n_arcs, c->neg_tab, c->n_nodes, seed, m, c->dscratch, c->stream),
       "line_eval_loss_noalloc");
    CK(cudaMemcpyAsync(out_host, c->dscratch, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
       "line_eval_loss_noalloc");
    CK(cudaStreamSynchronize(c->stream), "line_eval_loss_noalloc");
    return LINE_OK;
}

line_status line_get_stats(line_ctx* c, line_stats* out) {
    if (!c || !out) return LINE_ERR_ARG;
    out->update_launches = c->times.update_launches;
    out->update_ms = c->times.update_ms;
    out->update_samples = c->times.update_samples;
    out->prepass_launches = c->times.prepass_launches;
    out->prepass_ms = c->times.prepass_ms;
    out->total_ms = c->total_ms;
    out->total_samples = c->total_samples;
    return LINE_OK;
}

line_status line_reset_stats(line_ctx* c) {
    if (!c) return LINE_ERR_ARG;
    c->times = TrainTimes{};
    c->total_ms = 0;
    c->total_samples = 0;
    return LINE_OK;
}

line_status line_synchronize(line_ctx* c) {
    line_status st = enter(c);
    if (st) return st;
    CK(cudaStreamSynchronize(c->stream), "line_synchronize");
    return LINE_OK;
}

line_status line_debug_wait_timeout(line_ctx* c, int64_t spin_limit) {
    line_status st = enter(c);
    if (st) return st;
    if (spin_limit < 1 || spin_limit > (1ll << 24)) return fail(c, LINE_ERR_ARG, "line_debug_wait_timeout: spin_limit out of range");
    CK(debug_wait(c->flag, spin_limit, c->status, c->stream), "debug wait");
    return check_status(c, "line_debug_wait_timeout", /*timeout_sticky=*/false);
}

}  // extern "C"
