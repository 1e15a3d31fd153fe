// Autotuner of the training launch configuration: times short training runs
// of each candidate (gather warps per block, batches per pre-pass chunk,
// schedule, and optionally the batch size) on scratch copies of the tables,
// and returns the fastest.  Each candidate trains an untimed window of
// samples, then is timed on the following window (fresh rows, as in
// training).  The caller's tables are not modified.
#include <cstring>
#include <vector>

#include "context.cuh"

using namespace line;

extern "C" {

line_status line_autotune(line_ctx* c, int order, int dim, int K, const line_lr* lr, const line_tune_opts* topts,
                          line_train_opts* io, double* best_rate) {
    NvtxRange nvtx("line_autotune");
    line_status st = enter(c);
    if (st) return st;
    if (!c->has_graph) return fail(c, LINE_ERR_STATE, "line_autotune: no graph");
    if (order != 1 && order != 2) return fail(c, LINE_ERR_ARG, "line_autotune: order must be 1 or 2");
    if (!io || !lr) return fail(c, LINE_ERR_ARG, "line_autotune: null options");
    line_tune_opts to{};
    if (topts) to = *topts;
    // the tables the trials train: order `order`, or both orders
    std::vector<int> orders = to.both_orders ? std::vector<int>{1, 2} : std::vector<int>{order};
    for (int o : orders)
        if (!c->tab[o].ready || c->tab[o].dim != dim)
            return fail(c, LINE_ERR_STATE, "line_autotune: tables of order %d and dim %d not initialised", o, dim);
    if (to.n_batches < 0 || to.n_batches > 16 || (to.n_batches > 0 && !to.batches))
        return fail(c, LINE_ERR_ARG, "line_autotune: bad batch list");
    std::vector<int64_t> batches;
    for (int i = 0; i < to.n_batches; ++i) {
        if (to.batches[i] < 1 || to.batches[i] > (1 << 20)) return fail(c, LINE_ERR_ARG, "line_autotune: batch out of range");
        batches.push_back(to.batches[i]);
    }
    if (batches.empty()) batches.push_back(io->batch);
    // candidates
    struct Cand {
        int64_t batch;
        int wpb, cb, mode;
    };
    std::vector<Cand> cands;
    for (int64_t B : batches) {
        const int cb_auto = (int)std::max<int64_t>(1, ((int64_t)1 << 18) / B);
        for (int cb : {cb_auto, std::max(1, cb_auto / 2)}) {
            for (int wpb : {1, 2, 4}) cands.push_back({B, wpb, cb, LINE_MODE_BATCHED});
            if (to.try_persistent) cands.push_back({B, 0, cb, LINE_MODE_PERSISTENT});
            if (cb_auto == 1) break;
        }
    }
    // scratch copies of the tables: the trials train on them
    struct Saved {
        int order;
        void* U;
        void* C;
    };
    std::vector<Saved> saved;
    std::vector<void*> scratch;
    cudaError_t e = cudaSuccess;
    for (int o : orders) {
        Tables& t = c->tab[o];
        const size_t bytes = (size_t)c->n_nodes * dim * elem_size(t.dtype);
        void* sU = nullptr;
        void* sC = nullptr;
        if (e == cudaSuccess) e = cudaMalloc(&sU, bytes);
        if (sU) scratch.push_back(sU);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sU, t.U, bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess && t.C) e = cudaMalloc(&sC, bytes);
        if (sC) scratch.push_back(sC);
        if (e == cudaSuccess && t.C) e = cudaMemcpyAsync(sC, t.C, bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) break;
        saved.push_back({o, t.U, t.C});
        t.U = sU;
        t.C = sC;
    }
    auto restore = [&] {
        cudaStreamSynchronize(c->stream);
        for (const Saved& sv : saved) {
            c->tab[sv.order].U = sv.U;
            c->tab[sv.order].C = sv.C;
        }
        for (void* p : scratch) cudaFree(p);
    };
    if (e != cudaSuccess) {
        restore();
        return cuda_fail(c, e, "line_autotune: scratch tables");
    }
    const TrainTimes saved_times = c->times;
    const double saved_ms = c->total_ms;
    const uint64_t saved_samples = c->total_samples;
    double best = -1.0;
    Cand win = cands[0];
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (const Cand& cd : cands) {
        if (e != cudaSuccess || st != LINE_OK) break;
        line_train_opts o = *io;
        o.batch = cd.batch;
        o.warps_per_block = cd.wpb;
        o.chunk_batches = cd.cb;
        o.mode = cd.mode;
        o.timing = 0;
        o.graph = 1;
        // at least four chunks, or the requested count, rounded to whole batches
        uint64_t n = to.trial_samples ? to.trial_samples : (uint64_t)4 * cd.cb * cd.batch;
        n = (n + cd.batch - 1) / cd.batch * cd.batch;
        // one untimed run (allocations, graph capture), then the timed one on
        // the next n samples: a repeat of the same samples would find their
        // rows in L2 and rate every candidate above what training sees
        const uint64_t off0 = io->sample_offset;
        auto trial = [&](uint64_t offset) {
            o.sample_offset = offset;
            return to.both_orders ? line_train_orders(c, dim, K, lr, n, 0x5EED, &o)
                                  : line_train_steps(c, order, dim, K, lr, n, 0x5EED, &o);
        };
        st = trial(off0);
        if (st) break;
        if ((e = cudaEventRecord(e0, c->stream)) != cudaSuccess) break;
        st = trial(off0 + n);
        if (st) break;
        if ((e = cudaEventRecord(e1, c->stream)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double rate = ms > 0.0f ? (double)n * orders.size() / (ms * 1e-3) : 0.0;
        if (rate > best) {
            best = rate;
            win = cd;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    restore();
    c->times = saved_times;
    c->total_ms = saved_ms;
    c->total_samples = saved_samples;
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(c, e, "line_autotune");
    io->batch = win.batch;
    io->warps_per_block = win.wpb;
    io->chunk_batches = win.cb;
    io->mode = win.mode;
    io->graph = 1;
    if (best_rate) *best_rate = best;
    return LINE_OK;
}

}  // extern "C"
