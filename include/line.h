/*
 * line.h - C ABI of the GB300 (sm_103a) LINE training library.
 *
 * The library implements, on one GPU, the LINE training step that NOMAD
 * (arXiv 2604.09419) distributes over CPU clusters:
 *   - weight-proportional arc (positive pair) selection - Algorithm 3, the
 *     discrete distribution over E_p / ||E_p||;
 *   - K negatives per positive from q(v) = d(v)^0.75 / sum_x d(x)^0.75 -
 *     Section IV-A, Eq. 1 (d = weighted out-degree);
 *   - per pair the gradient scalar g = eta(1 - sigma(U[u].C[v])) or
 *     g = -eta alpha_neg sigma(U[u].C[v-]) - Algorithm 1 - and the
 *     LineUpdate of Eq. 2-3;
 *   - minibatch-synchronous semantics: all contributions to a row within a
 *     batch are computed from the batch-start tables and summed before being
 *     applied once, as the owner applies the summed remote deltas of Eq. 4.
 *     The sum runs over a sorted segmented reduction in a fixed order, so
 *     results are bitwise reproducible;
 *   - alternatively, the local path of Algorithm 1 (LineUpdate applied pair
 *     after pair) run by lock-free concurrent workers (LINE_MODE_HOGWILD);
 *   - positive pairs from weighted random walks (Algorithms 2-3, the Local
 *     variant of Section IV-C; opts.walk_length, opts.window, opts.walk_reuse);
 *   - link-prediction AUC and the LINE loss for reporting, and an MLP that
 *     predicts the rows of new nodes from their degree and neighbours (the
 *     line_mlp_* calls).
 *
 * Every draw is a Philox4x32-10 output (Salmon et al., SC'11) at counter
 * (t_lo, t_hi, call, domain) under key (seed_lo, seed_hi); t is the global
 * sample index, call 0 draws the arc and calls 1..K the negatives, domain 0
 * is training, 1 table initialisation, 3 the loss evaluation, 7 the MLP and
 * 8 the walks.  A draw maps its words (w0, w1, w2)
 * through an alias table: i = mulhi64(w1:w0, n), k = w2 < thr[i] ? i : alias[i].
 *
 * Conventions
 *   - Every call returns a line_status.  After LINE_ERR_CUDA or
 *     LINE_ERR_TIMEOUT the context is sticky-errored: later calls return
 *     LINE_ERR_STATE until line_destroy.  line_last_error() describes the
 *     first failure.
 *   - All GPU work is enqueued on the stream given to line_create and is
 *     stream ordered.  Calls that return a value to the host (train, eval,
 *     get_alias with host buffers, get_stats) synchronise that stream.
 *   - Pointers named "buffer" may be device memory or host memory (the
 *     library copies with unified addressing); the caller owns them and may
 *     free them when the call returns.
 *   - The library owns every device allocation it makes (graph copy, alias
 *     tables, embedding tables, scratch) and frees them in line_destroy.
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef LINE_H
#define LINE_H

#include <stdint.h>

#if defined(__GNUC__)
#define LINE_API __attribute__((visibility("default")))
#else
#define LINE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct line_ctx line_ctx;

typedef enum {
    LINE_OK = 0,
    LINE_ERR_ARG = -1,      /* invalid argument; nothing was enqueued */
    LINE_ERR_OOM = -2,      /* a device allocation failed */
    LINE_ERR_CUDA = -3,     /* a CUDA call or kernel failed (sticky) */
    LINE_ERR_TIMEOUT = -4,  /* a device wait exceeded its spin limit (sticky) */
    LINE_ERR_STATE = -5,    /* call out of order (no graph / no tables) or sticky error */
    LINE_ERR_VALIDATE = -6  /* input graph or table failed validation */
} line_status;

enum { LINE_DTYPE_F32 = 0, LINE_DTYPE_BF16 = 1 };
enum { LINE_TABLE_EDGE = 0, LINE_TABLE_NEG = 1 };
enum { LINE_WHICH_U = 0, LINE_WHICH_C = 1 };
enum { LINE_MODE_BATCHED = 0, LINE_MODE_PERSISTENT = 1, LINE_MODE_HOGWILD = 2 };
enum { LINE_SCORE_DOT = 0, LINE_SCORE_COSINE = 1 };

/* Graph as directed arcs (an undirected edge is two arcs), Section II / V-A.
 * src, dst: n_arcs int32 node ids in [0, n_nodes); src must be
 * non-decreasing (CSR order).  w: n_arcs positive finite weights, or NULL
 * for unit weights.  The three are buffers (device or host); they are read
 * during line_build_alias only. */
typedef struct {
    int64_t n_nodes;
    int64_t n_arcs;
    const int32_t* src;
    const int32_t* dst;
    const float* w;
} line_graph_desc;

/* Learning rate per batch (Section V-A: eta = 0.025):
 * schedule 0: eta_b = lr0;  schedule 1: eta_b = lr0 * max(1 - t0/T, floor_frac)
 * with t0 the first global sample index of the batch and T = total
 * (total == 0 means sample_offset + n_samples of the call). */
typedef struct {
    double lr0;
    int schedule;
    double floor_frac;
    uint64_t total;
} line_lr;

/* Options of line_train_steps.  Fill with line_train_opts_default(). */
typedef struct {
    int64_t batch;           /* B: samples per minibatch (Algorithm 1), 1..1048576 */
    double lambda;           /* weight decay lambda of Eq. 2-3 (>= 0) */
    double alpha_neg;        /* negative weight alpha_neg of Algorithm 1 */
    uint64_t sample_offset;  /* global index of the first sample; batches start here */
    int mode;                /* LINE_MODE_BATCHED or LINE_MODE_PERSISTENT (minibatch-synchronous,
                                Eq. 4, deterministic), or LINE_MODE_HOGWILD (see below) */
    int64_t spin_limit;      /* bound on every device wait loop (iterations); <= 0: default */
    int chunk_batches;       /* batches per pre-pass chunk; 0: automatic */
    int warps_per_block;     /* 0: automatic */
    int timing;              /* 1: time the training kernels with CUDA events (line_get_stats) */
    int graph;               /* 1: batched mode replays each full chunk's launches from a
                                captured CUDA graph (same results); 0: direct launches */
    int walk_length;         /* L > 0: positive pairs from random walks of L steps
                                (Algorithms 2-3, see line_sample_walk_debug); 0: arcs
                                drawn by weight (Eq. 1).  At most 1024. */
    int window;              /* W: pair window of the walk sampler, 1 <= W <= L */
    int hogwild_workers;     /* LINE_MODE_HOGWILD: samples in flight at once (>= 0; 0: one
                                resident wave of the GPU, one worker per lane group) */
    int walk_reuse;          /* r: passes over each walk's pairs, 1..1024 (0 means 1): sample t
                                takes pair t mod P of walk t / (r P) - a single-device form of
                                the Reuse-Spill variant (§IV-C) */
} line_train_opts;

/* LINE_MODE_HOGWILD: the local path of Algorithm 1 - LineUpdate applied pair
 * after pair, at once, with no minibatch.  For each sample in order and each
 * of its pairs (u, v), (u, n_1) .. (u, n_K) in order: x = U[u], c = Ctx[y]
 * (both before the call), s = x . c, g = eta (1 - sigma(s)) or
 * -eta alpha_neg sigma(s), U[u] <- x + (g c - eta lambda x), then
 * Ctx[y] <- c + (g x - eta lambda c).  eta is the schedule's value at the
 * first sample of the sample's block of opts.batch samples.  Workers run
 * samples concurrently on the shared tables without locks (Hogwild): a
 * worker sees other workers' rows as they are when it loads them, and adds
 * its changes to the rows with atomic read-modify-writes, so no worker's
 * change is overwritten by another's (the context row's change after each
 * call, U[u]'s net change after the sample's last call; BF16 tables add the
 * change plus uniform noise of one unit in the last place, rounded to
 * nearest).  With more than one worker the order of the additions, hence the
 * result, is not deterministic; hogwild_workers = 1 is the sequential
 * per-pair SGD.  Samples (arcs or walk pairs, negatives) are the same as in
 * the other modes. */

/* Counters of the training calls since the last line_reset_stats.  Launch
 * and sample counts are kept on every call (a replayed CUDA graph counts the
 * kernels it holds; line_train_orders counts both orders); the times only
 * with opts.timing == 1. */
typedef struct {
    int64_t update_launches;   /* launches of the row-update kernels (gather, apply, persistent, Hogwild) */
    double update_ms;          /* their summed CUDA-event time (opts.timing; not for line_train_orders) */
    uint64_t update_samples;   /* samples those launches processed */
    int64_t prepass_launches;  /* sampling + sort + segment launches */
    double prepass_ms;         /* (opts.timing; not for line_train_orders) */
    double total_ms;           /* event time of whole training calls (opts.timing) */
    uint64_t total_samples;    /* samples of those calls (opts.timing) */
} line_stats;

LINE_API void line_train_opts_default(line_train_opts* opts);
LINE_API const char* line_status_string(line_status s);

/* Create a context on CUDA device `device`; all work goes to `cuda_stream`
 * (a cudaStream_t, NULL for the legacy default stream).  *out receives the
 * context or NULL on failure.  No paper counterpart: the context holds what
 * one NOMAD process keeps in memory (its graph partition, distributions and
 * embedding rows, Algorithm 1's inputs), here for the whole graph on one GPU.
 * Errors: LINE_ERR_ARG (no such device, out NULL), LINE_ERR_CUDA. */
LINE_API line_status line_create(line_ctx** out, int device, void* cuda_stream);
LINE_API void line_destroy(line_ctx* ctx);
LINE_API const char* line_last_error(const line_ctx* ctx);

/* Copy the graph and build both alias tables on the GPU (Eq. 1 and
 * Algorithm 3).  Weights x (arc weights for the edge table; d(v)^0.75 for
 * the negative table, d summed over v's arcs in arc order, d^0.75 computed
 * as sqrt(d)*sqrt(sqrt(d))) are normalised in FP64: W is the sum of x in a
 * fixed order (blocks of 1024 reduced by halving strides, recursively),
 * S = n*2^32/W, m_i = floor(x_i*S), and the remainder D = n*2^32 - sum(m) is
 * spread round robin over x_i > 0 (D > 0) or taken from the first |D| items
 * with m_i >= 1 (D < 0).  Light buckets (m < 2^32) are paired with heavy
 * items (m > 2^32) by the sweep rule: heavy items in index order top up the
 * lights in index order, a heavy item whose remaining mass r falls below
 * 2^32 becomes a light bucket with thr = r topped up by the next heavy one.
 * Replaces any previous graph.  Embedding tables (and the warm-start MLP)
 * are kept when the new graph has the same n_nodes - so training can
 * continue on a changed edge set - and dropped otherwise.  The library
 * keeps its own device copy of src, dst and w (4 bytes per arc each; w only
 * when given), the alias tables and the weighted degrees; per-node arc
 * offsets (8 bytes per node) and the walk sampler's weight sums (8 bytes per
 * arc) are added on first use.  A later graph reuses these buffers (and the
 * build's FP64 scratch, 8 bytes per arc or node) when they are large enough;
 * they are freed by line_destroy.
 * Errors: LINE_ERR_ARG (sizes), LINE_ERR_VALIDATE (unsorted src, ids out of
 * range, non-positive or non-finite weights, a node set with no positive
 * weight), LINE_ERR_OOM. */
LINE_API line_status line_build_alias(line_ctx* ctx, const line_graph_desc* g);

/* Node and arc counts of the current graph (host pointers, either may be
 * NULL).  No paper counterpart (bookkeeping).  Errors: LINE_ERR_STATE (no
 * graph). */
LINE_API line_status line_get_graph_info(line_ctx* ctx, int64_t* n_nodes, int64_t* n_arcs);

/* Export an alias table (LINE_TABLE_EDGE: n_arcs entries; LINE_TABLE_NEG:
 * n_nodes entries) into two uint32 buffers thr[] and alias[].  These are the
 * samplers of the edge distribution of Algorithm 3 and of q(v) of Eq. 1
 * (Section IV-A); the paper names only the distributions, the alias form is
 * this library's (see line_build_alias).  Errors: LINE_ERR_ARG (bad table,
 * NULL buffer), LINE_ERR_STATE (no graph). */
LINE_API line_status line_get_alias(line_ctx* ctx, int table, uint32_t* thr, uint32_t* alias);

/* Write the draws of samples t0 .. t0+count-1 in `domain` as int32 records
 * out[count][K+2] = (u, v, n_1 .. n_K) (a buffer). */
LINE_API line_status line_sample_debug(line_ctx* ctx, int K, uint64_t seed, uint32_t domain, uint64_t t0,
                              int64_t count, int32_t* out);

/* Walk sampler (Algorithms 2-3, the local walk of one partition): write the
 * records of samples t0 .. t0+count-1 as out[count][K+2] = (u, v, n_1 .. n_K)
 * (a host or device buffer).  Sample t takes pair t mod P of walk t / P,
 * P = L W - W (W - 1) / 2.  Walk wk starts at the arc drawn from the edge
 * alias table with draw (wk, call 0) of domain 8: nodes[0] = src,
 * nodes[1] = dst.  Step i = 1 .. L-1 leaves x = nodes[i] by the first of its
 * arcs e whose running FP64 weight sum cw[e] (arc order) exceeds
 * u * cw[last arc of x], u = ((w1:w0) >> 11) 2^-53 from words w0, w1 of draw
 * (wk, call i) of domain 8 (the last arc if none does); a node without
 * out-arcs steps back to nodes[i-1].  The pairs of a walk are
 * (nodes[i], nodes[i+k]), i = 0 .. L-1, k = 1 .. W, i + k <= L, in (i, k)
 * order.  Negatives are the edge sampler's (domain 0, calls 1..K at counter
 * t).  With reuse r > 1 each walk's pairs serve r passes in a row: sample
 * t takes pair t mod P of walk t / (r P).  The first call on a graph builds
 * the per-node arc offsets and weight sums (12 bytes per arc with the kept
 * weights, 8 per node); their memory is reused by later graphs that fit and
 * freed by line_destroy.
 * Errors: LINE_ERR_ARG (K, count, not 1 <= W <= L <= 1024, or reuse
 * outside 1..1024),
 * LINE_ERR_STATE (no graph). */
LINE_API line_status line_sample_walk_debug(line_ctx* ctx, int K, uint64_t seed, int walk_length, int window,
                                            int reuse, uint64_t t0, int64_t count, int32_t* out);

/* (Re)create the tables of one order: order 1 has U only (the context of a
 * pair is U, first-order proximity), order 2 has U and C (second order).
 * U[i][k] = ((w >> 8) - 2^23) * 2^-24 / dim with w = word (k mod 4) of the
 * draw at counter (i_lo, i_hi, k/4, 1): uniform on [-0.5/dim, 0.5/dim);
 * C = 0.  dim in {16, 32, 64, 128, 256}; dtype LINE_DTYPE_F32 or
 * LINE_DTYPE_BF16 (storage; arithmetic is FP32, BF16 write-back uses
 * stochastic rounding: 16 random bits added below the BF16 mantissa, then
 * truncation; the 64 bits of values 4k..4k+3 of a row written by the batch
 * starting at sample t0 are two MurmurHash3 fmix32 words, of b and b + 1,
 * b = lo32(SplitMix64 output of seed ^ t0 0x9E3779B97F4A7C15) +
 * (2 row + table) 0x9E3779B1 + 2k, table 0 for U and 1 for C).  Re-creating
 * tables reuses their device memory when it is large enough. */
LINE_API line_status line_init_embeddings(line_ctx* ctx, int order, int dim, int dtype, uint64_t seed);

/* Train n_samples samples (global indices sample_offset .. +n_samples-1) of
 * order 1 or 2 with K negatives (0..32) per positive, minibatch-synchronous
 * (see the file comment).  Splitting a run at a multiple of opts.batch from
 * its first offset, with the same lr->total, gives bitwise identical tables.
 * Synchronises the stream at the end to read the device status word.
 * Errors: LINE_ERR_ARG, LINE_ERR_STATE (no graph or tables of that order and
 * dim), LINE_ERR_TIMEOUT (persistent mode: a dependency wait exceeded
 * opts.spin_limit), LINE_ERR_CUDA. */
LINE_API line_status line_train_steps(line_ctx* ctx, int order, int dim, int K, const line_lr* lr,
                             uint64_t n_samples, uint64_t seed, const line_train_opts* opts);

/* Train the order-1 and the order-2 tables (both created with `dim`) on
 * the same samples, concurrently: the two runs are independent (separate
 * tables), so the call gives bitwise the same tables as
 * line_train_steps(order 1) followed by line_train_steps(order 2) with the
 * same arguments, while the GPU overlaps one run's latency-bound phases with
 * the other's.  The order-1 run uses a second stream and workspace owned by
 * the context; the two runs are issued in alternate slices of about 2^24
 * samples, so that a long call keeps work of both orders queued.  Work after
 * the call on the context's stream follows both runs.  opts.timing times the call as a whole (total_ms, total_samples =
 * 2 n_samples) and not per kernel.  Errors: as line_train_steps. */
LINE_API line_status line_train_orders(line_ctx* ctx, int dim, int K, const line_lr* lr, uint64_t n_samples,
                                       uint64_t seed, const line_train_opts* opts);

/* Search space of line_autotune. */
typedef struct {
    const int64_t* batches;  /* candidate batch sizes (a host array), or NULL: keep io->batch */
    int n_batches;           /* 0..16 */
    uint64_t trial_samples;  /* samples per timed trial; 0: four pre-pass chunks */
    int try_persistent;      /* 1: also time the persistent schedule */
    int both_orders;         /* 1: time line_train_orders on both orders' tables (order ignored) */
} line_tune_opts;

/* Autotuner of the launch configuration (not in the paper, whose CPU code
 * has no such knobs): for every candidate - gather warps per block (1, 2,
 * 4), batches per pre-pass chunk (about 2^18 samples, and half that), the
 * batched schedule with graph replay (and the persistent one if asked), each
 * listed batch size - it runs an untimed training run of trial_samples from
 * io->sample_offset and a timed one of the next trial_samples (fresh rows,
 * as training meets them) on scratch copies of the order's tables, and
 * writes the
 * fastest into *io (batch, warps_per_block, chunk_batches, mode, graph; the
 * other fields of *io are used as given).  With topts->both_orders the trials
 * train both orders concurrently (line_train_orders) and the rate counts both.  The tables, the statistics and
 * the learning-rate state of the caller are unchanged.  Changing the batch
 * size changes the results (minibatch semantics): list batch sizes only when
 * that is acceptable.  *best_rate (if not NULL): the winner's samples/s.
 * Errors: as line_train_steps; LINE_ERR_OOM if the scratch tables do not fit. */
LINE_API line_status line_autotune(line_ctx* ctx, int order, int dim, int K, const line_lr* lr,
                                   const line_tune_opts* topts, line_train_opts* io, double* best_rate);

/* Copy a whole table (n_nodes x dim, row-major) into `dst` (a buffer) as
 * dst_dtype (F32, or BF16 when the table is BF16).  These are the outputs U
 * and C of Algorithm 1 (the trained embeddings); the call itself has no
 * paper counterpart.  Errors: LINE_ERR_ARG, LINE_ERR_STATE (no such table). */
LINE_API line_status line_get_embeddings(line_ctx* ctx, int order, int which, void* dst, int dst_dtype);

/* Overwrite rows of a table from `src` (a buffer of n_rows x dim values of
 * src_dtype).  rows: n_rows int32 row ids (a buffer), or NULL for rows
 * 0..n_rows-1.  F32 into a BF16 table rounds to nearest even.  Used for
 * warm starts and checkpoint restore.  No paper counterpart: the paper's
 * rows start only from the random initialisation of Algorithm 1.
 * Errors: LINE_ERR_ARG (bad arguments, or a row id out of range: that row is
 * skipped, the others are written), LINE_ERR_STATE (no such table),
 * LINE_ERR_OOM. */
LINE_API line_status line_set_embeddings(line_ctx* ctx, int order, int which, const void* src, int src_dtype,
                                const int32_t* rows, int64_t n_rows);

/* Negative-sampling LINE loss over the first m samples of draw domain 3:
 * L = -sum_t [log sigma(s+) + sum_j log sigma(-s-_j)], s = U[u].Ctx[y]
 * computed in FP64 from the stored values, summed in a fixed order.
 * Result in *out_host (host pointer). */
LINE_API line_status line_eval_loss(line_ctx* ctx, int order, int K, uint64_t seed, int64_t m, double* out_host);

/* Link-prediction AUC: held-out edges against non-edges (the paper's own
 * quality measure, node classification in §V-C, needs node labels).
 * orders: bit mask of the tables to use - 1 the order-1 U
 * table, 2 the order-2 U table, 3 both.  With z(x) the concatenation over
 * those orders of U_o[x], a pair (u, v) scores, in FP32,
 *   LINE_SCORE_DOT:    z(u).z(v);
 *   LINE_SCORE_COSINE: the cosine of the concatenations of U_o[u] / |U_o[u]|
 *     and U_o[v] / |U_o[v]| (an all-zero row gives a zero block; a zero
 *     concatenation scores 0).
 * AUC = (#(neg < pos) + #(neg == pos) / 2) / (n_pos n_neg) over all
 * (positive, negative) pairs of scores, counted exactly in integers.
 *   pos_src/pos_dst: n_pos >= 1 node ids of the positive pairs (held-out
 *     edges); neg_src/neg_dst: n_neg >= 1 node ids of the negative pairs;
 *     buffers (host or device), read during the call only.
 *   scores_out: NULL, or a buffer of n_pos + n_neg floats (positives first).
 *   counts_out: NULL, or a host array of 2: {#(neg < pos), #(neg == pos)}.
 *   auc_out: host pointer.
 * Errors: LINE_ERR_ARG (bad mask or score, counts, null pointers, or a node
 * id out of range), LINE_ERR_STATE (a requested order has no tables),
 * LINE_ERR_VALIDATE (a score is NaN: non-finite table values), LINE_ERR_OOM,
 * LINE_ERR_CUDA.  Allocates scratch for the pairs per call; synchronises. */
LINE_API line_status line_eval_auc(line_ctx* ctx, int orders, int score, const int32_t* pos_src, const int32_t* pos_dst,
                                   int64_t n_pos, const int32_t* neg_src, const int32_t* neg_dst, int64_t n_neg,
                                   float* scores_out, uint64_t* counts_out, double* auc_out);

/* ------------------------------------------------------------------------
 * Warm start of new or held-out nodes.  Not in the paper, whose rows all
 * start from a random draw (Algorithm 1): a two-layer MLP regresses trained U
 * rows of one order on inputs every node has, and its predictions initialise
 * the rows of nodes LINE has not trained; plain LINE refinement follows.
 * For the table dimension d and hidden width H, P = d + 1 rounded up to a
 * multiple of 16:
 *   x = [log(1 + d_w(v)), mean of U[w] over arcs v -> w with known[w],
 *        0 ... ]                                     (d_w: weighted out-degree)
 *   a = W1 x + b1, h = GELU(a) = a/2 (1 + erf(a / sqrt 2)), y = W2 h + b2
 *   L = sum over a minibatch of B nodes of |y - U[v]|^2 / (B d)
 * Parameters, flat FP32 in this order: W1 (H x P, row-major), b1 (H),
 * W2 (d x H), b2 (d).  Optimiser: Adam with bias correction (beta1 0.9,
 * beta2 0.999, eps 1e-8).  The activations x and h are stored as
 * act_dtype (F32, or BF16 rounded to nearest even); sums are FP32 in a fixed
 * order, so results are bitwise reproducible.  Initial weights: Philox
 * domain 7, call 1, counter = flat index: u = ((w0 >> 8) - 2^23) 2^-23,
 * W1 = u / sqrt(d + 1) on the d + 1 used columns (0 on padding), W2 =
 * u / sqrt(H), biases 0.  Minibatch sample j of global step s is
 * nodes[mulhi64(w1:w0, n)] of the Philox draw of domain 7, call 0, counter
 * s B + j.  One MLP per context; line_build_alias with a different n_nodes
 * discards it.
 * ------------------------------------------------------------------------ */

/* Create (or replace) the MLP for the U table of `order` (which must exist),
 * hidden width 1..4096, activations act_dtype, initial weights from `seed`.
 * Replacing an MLP of the same order, width, activation type and node count
 * keeps its device memory; weights, optimiser state and inputs start over
 * either way.  Errors: LINE_ERR_ARG, LINE_ERR_STATE (no graph or tables),
 * LINE_ERR_OOM. */
LINE_API line_status line_mlp_create(line_ctx* ctx, int order, int hidden, int act_dtype, uint64_t seed);

/* Compute the inputs x of every node from the current U table.  known: a
 * buffer of n_nodes bytes, non-zero where the node's row is a trained
 * embedding (neighbours that are not known are left out of the mean). */
LINE_API line_status line_mlp_features(line_ctx* ctx, const uint8_t* known);

/* Compute the inputs of the nodes rows[0 .. n_rows) only (a buffer of node
 * ids, which may repeat), from the current graph and U table - for a sample
 * of nodes to fit on, or for nodes that joined later; the other nodes'
 * inputs are unchanged (zero until computed: line_mlp_create clears them).
 * A node's inputs are the same bits whether computed here or by
 * line_mlp_features.  Errors: LINE_ERR_ARG (an id out of range; nothing is
 * computed), LINE_ERR_STATE. */
LINE_API line_status line_mlp_features_rows(line_ctx* ctx, const uint8_t* known, const int32_t* rows,
                                            int64_t n_rows);

/* Copy the inputs (n_nodes x P) as FP32 into `out` (a buffer). */
LINE_API line_status line_mlp_get_features(line_ctx* ctx, float* out);

/* Number of parameters in *n_params (if not NULL) and, if `out` is not
 * NULL, a copy of them (a buffer of n_params floats). */
LINE_API line_status line_mlp_get_params(line_ctx* ctx, float* out, int64_t* n_params);

/* Overwrite the parameters from `in` (a buffer of n_params floats) and
 * restart the optimiser state (moments zero, step count 0). */
LINE_API line_status line_mlp_set_params(line_ctx* ctx, const float* in);

/* Loss and gradient of the minibatch rows[0 .. n_rows) (a buffer of node
 * ids, 1 <= n_rows <= 65536) at the current parameters, targets the current
 * U rows; no update.  grads_out: NULL or a buffer of n_params floats;
 * loss_out: NULL or a host pointer.  Needs the rows' inputs (line_mlp_features or
 * line_mlp_features_rows). */
LINE_API line_status line_mlp_grad(line_ctx* ctx, const int32_t* rows, int64_t n_rows, float* grads_out,
                                   double* loss_out);

/* `steps` Adam steps with learning rate lr on minibatches of `batch` nodes
 * (1..65536) drawn from nodes[0 .. n) (a buffer), global steps
 * step_offset .. step_offset + steps - 1; targets the current U rows.
 * losses_out: NULL or a host array of `steps` doubles, each step's loss
 * before its update.  Needs the nodes' inputs (line_mlp_features or
 * line_mlp_features_rows).  Node ids out of range:
 * LINE_ERR_ARG (the step uses row 0 instead). */
LINE_API line_status line_mlp_train(line_ctx* ctx, const int32_t* nodes, int64_t n, int64_t steps, int64_t batch,
                                    double lr, uint64_t seed, uint64_t step_offset, double* losses_out);

/* Predictions y for the nodes rows[0 .. n_rows) (a buffer).  y_out NULL:
 * written into those rows of the U table (BF16 tables round to nearest
 * even) - the warm start; otherwise a buffer of n_rows x d floats and the
 * table is untouched.  Needs the rows' inputs (line_mlp_features or
 * line_mlp_features_rows). */
LINE_API line_status line_mlp_predict(line_ctx* ctx, const int32_t* rows, int64_t n_rows, float* y_out);

/* Largest m accepted by line_eval_loss_noalloc. */
#define LINE_NOALLOC_MAX_SAMPLES (1 << 20)

/* line_eval_loss without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc while they run - for instance a service that reserved all device
 * memory for its tables up front and must not grow its footprint, or a
 * latency-bound loop in which cudaMalloc/cudaFree would synchronise the
 * device.  The per-sample terms and the partial sums live in one fixed
 * array of LINE_NOALLOC_MAX_SAMPLES + 1024 doubles (8 MiB + 8 KiB) that every
 * GPU loading this library holds until the process exits; the result is the
 * same as line_eval_loss.  m must be 1..LINE_NOALLOC_MAX_SAMPLES, otherwise
 * LINE_ERR_ARG and nothing runs.  line_create looks up the array's device
 * address on its device (under lazy module loading that first look-up loads
 * the array and may allocate it), so this call itself allocates nothing.  The
 * call ends by copying the result to the host and synchronising the
 * context's stream: it must not be made while that stream is being captured
 * into a CUDA graph.  All calls, from every context, share
 * the one array: calls whose GPU work overlaps (different streams or
 * contexts on the same device) race and give wrong results; calls ordered on
 * one stream are safe, and no state carries over from one call to the next.
 * Result in *out_host (host pointer). */
LINE_API line_status line_eval_loss_noalloc(line_ctx* ctx, int order, int K, uint64_t seed, int64_t m,
                                            double* out_host);

LINE_API line_status line_get_stats(line_ctx* ctx, line_stats* out);
LINE_API line_status line_reset_stats(line_ctx* ctx);

/* Wait for all work of the context's stream. */
LINE_API line_status line_synchronize(line_ctx* ctx);

/* Exercise the bounded device wait: launches a kernel that waits on a flag
 * nothing sets, for at most spin_limit polls, and returns LINE_ERR_TIMEOUT
 * when the wait runs out (the context stays usable: this timeout is not
 * sticky).  Used by the failure-handling tests. */
LINE_API line_status line_debug_wait_timeout(line_ctx* ctx, int64_t spin_limit);

#ifdef __cplusplus
}
#endif

#endif /* LINE_H */
