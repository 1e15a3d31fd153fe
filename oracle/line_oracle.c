/*
 * FP64 serial CPU oracle for the LINE training step that NOMAD distributes
 * (arXiv 2604.09419).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the CPU-baseline leg of the benchmark call it; the library never does.
 * It shares no source with the CUDA path.
 *
 * What it computes, in the paper's notation:
 *   - negative distribution q(v) ∝ d(v)^0.75 with d the (weighted) out-degree
 *     (Section IV-A, Eq. 1);
 *   - weight-proportional edge selection (Algorithm 3, the discrete
 *     distribution over E_p / ||E_p||);
 *   - both as alias tables over exact integer masses;
 *   - the per-pair gradient scalars g = eta(1 - sigma(U[u].C[v])) and
 *     g = -eta alpha_neg sigma(U[u].C[v-]) (Algorithm 1);
 *   - the LineUpdate of Algorithm 1 / Eq. 2-3 with the per-batch delta
 *     accumulation of Eq. 4: every row's contributions within a batch are
 *     summed against the batch-start tables and applied once after the batch.
 *
 * Everything is plain loops in the order of the definitions; no blocking, no
 * fusion.  Build: gcc -O2 -ffp-contract=off -shared -fPIC.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As   */
/* Easy as 1, 2, 3", SC'11): 10 rounds of the 4x32 S-box, key bumped by the  */
/* Weyl constants between rounds.                                            */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One draw: counter (t_lo, t_hi, call, domain), key (seed_lo, seed_hi). */
static void draw_words(uint64_t seed, uint32_t domain, uint64_t t, uint32_t call, uint32_t w[4]) {
    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), call, domain};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, w);
}

/* Words of `count` consecutive draws t0 .. t0+count-1 of one (domain, call):
 * out[4 t + i] = word i of draw t. */
void orc_draw_words(uint64_t seed, uint32_t domain, uint32_t call, uint64_t t0, int64_t count, uint32_t* out) {
    for (int64_t t = 0; t < count; ++t) draw_words(seed, domain, t0 + (uint64_t)t, call, out + 4 * t);
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 weights.                                                            */
/* ------------------------------------------------------------------------ */

/* d(v)^0.75 written as sqrt(d) * sqrt(sqrt(d)): both square roots and the
 * product are correctly rounded, so the value is a function of d alone. */
static double pow075(double d) {
    if (d <= 0.0) return 0.0;
    double r = sqrt(d);
    return r * sqrt(r);
}

/* d(v) = sum of the weights of v's out-arcs (arcs in index order, left to
 * right), then x_v = d(v)^0.75.  Arcs must be grouped by src; only src and w
 * are read.  w == NULL means unit weights. */
int orc_neg_weights(int64_t n_nodes, int64_t n_arcs, const int32_t* src, const float* w, double* x_out) {
    for (int64_t v = 0; v < n_nodes; ++v) x_out[v] = 0.0;
    for (int64_t e = 0; e < n_arcs; ++e) {
        int32_t s = src[e];
        if (s < 0 || s >= n_nodes) return -1;
        x_out[s] += w ? (double)w[e] : 1.0;
    }
    for (int64_t v = 0; v < n_nodes; ++v) x_out[v] = pow075(x_out[v]);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Alias tables over exact integer masses.                                   */
/* ------------------------------------------------------------------------ */
#define ALIAS_BLOCK 1024
#define Q32 4294967296ull
#define THR_FULL 0xFFFFFFFFu

/* Fixed-order FP64 sum: blocks of 1024 consecutive values (zero padded),
 * each reduced by halving strides (v[i] += v[i + s] for s = 512..1); the
 * block sums are reduced the same way, recursively. */
double orc_fixed_sum(int64_t n, const double* x) {
    if (n <= 0) return 0.0;
    int64_t nb = (n + ALIAS_BLOCK - 1) / ALIAS_BLOCK;
    double* sums = (double*)malloc(sizeof(double) * (size_t)nb);
    double buf[ALIAS_BLOCK];
    for (int64_t b = 0; b < nb; ++b) {
        for (int i = 0; i < ALIAS_BLOCK; ++i) {
            int64_t j = b * ALIAS_BLOCK + i;
            buf[i] = j < n ? x[j] : 0.0;
        }
        for (int s = ALIAS_BLOCK / 2; s >= 1; s /= 2)
            for (int i = 0; i < s; ++i) buf[i] = buf[i] + buf[i + s];
        sums[b] = buf[0];
    }
    double r = nb == 1 ? sums[0] : orc_fixed_sum(nb, sums);
    free(sums);
    return r;
}

/* Integer masses m_i with sum exactly n * 2^32:
 *   W = fixed-order sum of x;  S = (n * 2^32) / W;  m_i = floor(x_i * S);
 *   D = n * 2^32 - sum(m).
 *   D > 0: round-robin +1 over the indices with x_i > 0 in increasing order
 *          (q = D / P added to all P of them, +1 more to the first D % P);
 *   D < 0: -1 to each of the first |D| indices with m_i >= 1.
 * Returns 0, or -1 if W is not positive and finite, -2 if |D| cannot be
 * absorbed. */
int orc_alias_masses(int64_t n, const double* x, uint64_t* m) {
    double W = orc_fixed_sum(n, x);
    if (!(W > 0.0) || !isfinite(W)) return -1;
    double S = ((double)n * 4294967296.0) / W;
    uint64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        double f = floor(x[i] * S);
        m[i] = (uint64_t)f;
        total += m[i];
    }
    int64_t D = (int64_t)((uint64_t)n * Q32 - total);
    if (D > 0) {
        int64_t P = 0;
        for (int64_t i = 0; i < n; ++i) P += x[i] > 0.0;
        int64_t q = D / P, r = D % P, rank = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (x[i] > 0.0) {
                m[i] += (uint64_t)(q + (rank < r ? 1 : 0));
                ++rank;
            }
        }
    } else if (D < 0) {
        int64_t need = -D;
        for (int64_t i = 0; i < n && need > 0; ++i) {
            if (m[i] >= 1) {
                m[i] -= 1;
                --need;
            }
        }
        if (need > 0) return -2;
    }
    return 0;
}

/* Sweep pairing of light buckets (m < 2^32) with heavy ones (m > 2^32): the
 * current heavy item donates to the lights in increasing index order; when
 * its remaining mass r drops below 2^32 its own bucket becomes a light one
 * with threshold r, topped up by the next heavy item.  Buckets with
 * m == 2^32, and the last heavy item, keep all their mass.
 * Draw: i = mulhi64(w1:w0, n); k = (w2 < thr[i]) ? i : alias[i]. */
int orc_alias_pair(int64_t n, const uint64_t* m, uint32_t* thr, uint32_t* alias) {
    int64_t* heavy = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t nh = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (m[i] == Q32) {
            thr[i] = THR_FULL;
            alias[i] = (uint32_t)i;
        } else if (m[i] > Q32) {
            heavy[nh++] = i;
        }
    }
    int rc = 0;
    if (nh > 0) {
        int64_t k = 0;
        uint64_t r = m[heavy[0]];
        for (int64_t l = 0; l < n && rc == 0; ++l) {
            if (m[l] >= Q32) continue;
            thr[l] = (uint32_t)m[l];
            alias[l] = (uint32_t)heavy[k];
            r -= Q32 - m[l];
            while (r < Q32) {
                if (k + 1 >= nh) { rc = -3; break; }
                thr[heavy[k]] = (uint32_t)r;
                alias[heavy[k]] = (uint32_t)heavy[k + 1];
                r = m[heavy[k + 1]] - (Q32 - r);
                ++k;
            }
        }
        if (rc == 0) {
            if (k != nh - 1 || r != Q32) rc = -4;
            thr[heavy[k]] = THR_FULL;
            alias[heavy[k]] = (uint32_t)heavy[k];
        }
    } else {
        for (int64_t i = 0; i < n; ++i)
            if (m[i] < Q32) rc = -5; /* lights without heavies: masses do not sum to n*2^32 */
    }
    free(heavy);
    return rc;
}

int orc_alias_build(int64_t n, const double* x, uint64_t* m_out, uint32_t* thr, uint32_t* alias) {
    int rc = orc_alias_masses(n, x, m_out);
    if (rc) return rc;
    return orc_alias_pair(n, m_out, thr, alias);
}

static inline uint32_t alias_draw(int64_t n, const uint32_t* thr, const uint32_t* alias,
                                  uint32_t w0, uint32_t w1, uint32_t w2) {
    uint64_t r64 = ((uint64_t)w1 << 32) | (uint64_t)w0;
    uint64_t i = (uint64_t)(((unsigned __int128)r64 * (unsigned __int128)(uint64_t)n) >> 64);
    return w2 < thr[i] ? (uint32_t)i : alias[i];
}

uint32_t orc_alias_draw(int64_t n, const uint32_t* thr, const uint32_t* alias,
                        uint32_t w0, uint32_t w1, uint32_t w2) {
    return alias_draw(n, thr, alias, w0, w1, w2);
}

/* ------------------------------------------------------------------------ */
/* Per-sample draws: sample t, call 0 draws the arc e (u = src[e],           */
/* v = dst[e]); calls 1..K draw the negatives from q (Algorithm 1, Eq. 1).   */
/* out[(t - t0) * (K + 2) + {0, 1, 1 + j}] = u, v, n_j.                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n_nodes, n_arcs;
    const int32_t* src;
    const int32_t* dst;
    const uint32_t* thr_e;
    const uint32_t* alias_e;
    const uint32_t* thr_n;
    const uint32_t* alias_n;
} orc_tables;

static void sample_one(const orc_tables* T, uint64_t seed, uint32_t domain, uint64_t t, int K, int32_t* rec) {
    uint32_t w[4];
    draw_words(seed, domain, t, 0, w);
    uint32_t e = alias_draw(T->n_arcs, T->thr_e, T->alias_e, w[0], w[1], w[2]);
    rec[0] = T->src[e];
    rec[1] = T->dst[e];
    for (int j = 1; j <= K; ++j) {
        draw_words(seed, domain, t, (uint32_t)j, w);
        rec[1 + j] = (int32_t)alias_draw(T->n_nodes, T->thr_n, T->alias_n, w[0], w[1], w[2]);
    }
}

int orc_sample(int64_t n_nodes, int64_t n_arcs, const int32_t* src, const int32_t* dst,
               const uint32_t* thr_e, const uint32_t* alias_e, const uint32_t* thr_n, const uint32_t* alias_n,
               uint64_t seed, uint32_t domain, uint64_t t0, int64_t count, int K, int32_t* out) {
    orc_tables T = {n_nodes, n_arcs, src, dst, thr_e, alias_e, thr_n, alias_n};
    for (int64_t i = 0; i < count; ++i) sample_one(&T, seed, domain, t0 + (uint64_t)i, K, out + i * (K + 2));
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Walk sampler: the positive pairs of a random walk (Algorithms 2-3, the    */
/* local walk of one partition).  Walk wk starts at an arc drawn by weight   */
/* (draw wk of domain 8, call 0): nodes[0] = src, nodes[1] = dst.  Step i    */
/* (i = 1 .. L-1) moves from x = nodes[i] to an out-neighbour drawn by arc   */
/* weight: with words (w0, w1) of draw wk, call i, domain 8,                 */
/* u = ((w1:w0) >> 11) 2^-53 and target = u * d(x), the first arc e of x     */
/* whose cumulative weight cw[e] > target (the last arc if none); a node     */
/* without out-arcs steps back to nodes[i-1].  The pairs of a walk are       */
/* (nodes[i], nodes[i+k]) for i = 0 .. L-1, k = 1 .. W, i + k <= L, in       */
/* (i, k) order: P = L W - W (W - 1) / 2 of them.  Sample t takes pair       */
/* t mod P of walk t / P; its negatives are the edge sampler's (domain 0,    */
/* calls 1..K at counter t).  With reuse r (a single-device form of the      */
/* Reuse-Spill variant, §IV-C), each walk's pairs serve r passes in a row:   */
/* sample t takes pair t mod P of walk t / (r P).                            */
/* ------------------------------------------------------------------------ */
#define WALK_DOMAIN 8u

/* cw[e] = sum of the weights of src[e]'s arcs up to and including e, FP64 in
 * arc order (src sorted). */
void orc_walk_cumw(int64_t n_arcs, const int32_t* src, const float* w, double* cw) {
    double run = 0.0;
    for (int64_t e = 0; e < n_arcs; ++e) {
        if (e == 0 || src[e] != src[e - 1]) run = 0.0;
        run += w ? (double)w[e] : 1.0;
        cw[e] = run;
    }
}

typedef struct {
    orc_tables T;
    const double* cw;
    int reuse;  /* passes over each walk's pairs (>= 1) */
} orc_walker;

static int64_t first_arc_of(const orc_tables* T, int32_t v) {
    int64_t lo = 0, hi = T->n_arcs;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (T->src[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int32_t walk_step(const orc_walker* W, int32_t x, int32_t prev, const uint32_t w[4]) {
    int64_t lo = first_arc_of(&W->T, x), hi = first_arc_of(&W->T, x + 1);
    if (lo == hi) return prev;  /* a dead end steps back */
    uint64_t r = (((uint64_t)w[1] << 32) | (uint64_t)w[0]) >> 11;
    double u = (double)r * (1.0 / 9007199254740992.0);
    double target = u * W->cw[hi - 1];
    /* the first arc whose cumulative weight exceeds the target, by scanning */
    for (int64_t e = lo; e < hi; ++e)
        if (W->cw[e] > target) return W->T.dst[e];
    return W->T.dst[hi - 1];
}

/* nodes[0 .. L] of walk wk */
static void walk_nodes(const orc_walker* W, uint64_t seed, uint64_t wk, int L, int32_t* nodes) {
    uint32_t w[4];
    draw_words(seed, WALK_DOMAIN, wk, 0, w);
    uint32_t e = alias_draw(W->T.n_arcs, W->T.thr_e, W->T.alias_e, w[0], w[1], w[2]);
    nodes[0] = W->T.src[e];
    nodes[1] = W->T.dst[e];
    for (int i = 1; i < L; ++i) {
        draw_words(seed, WALK_DOMAIN, wk, (uint32_t)i, w);
        nodes[i + 1] = walk_step(W, nodes[i], nodes[i - 1], w);
    }
}

int64_t orc_walk_pairs_per_walk(int L, int Wn) { return (int64_t)L * Wn - (int64_t)Wn * (Wn - 1) / 2; }

/* pair p of a walk as (i, k), by counting the pairs of each node in order */
static void walk_pair(int L, int Wn, int64_t p, int* i_out, int* k_out) {
    for (int i = 0; i < L; ++i) {
        int n = Wn < L - i ? Wn : L - i;
        if (p < n) { *i_out = i; *k_out = (int)p + 1; return; }
        p -= n;
    }
    *i_out = 0;
    *k_out = 1;
}

static void sample_walk_one(const orc_walker* W, uint64_t seed, uint64_t t, int K, int L, int Wn, int32_t* nodes,
                            int64_t* cached, int32_t* rec) {
    int64_t P = orc_walk_pairs_per_walk(L, Wn);
    uint64_t wk = t / ((uint64_t)P * (uint64_t)W->reuse);
    if (*cached != (int64_t)wk) { walk_nodes(W, seed, wk, L, nodes); *cached = (int64_t)wk; }
    int i, k;
    walk_pair(L, Wn, (int64_t)(t % (uint64_t)P), &i, &k);
    rec[0] = nodes[i];
    rec[1] = nodes[i + k];
    uint32_t w[4];
    for (int j = 1; j <= K; ++j) {
        draw_words(seed, 0, t, (uint32_t)j, w);
        rec[1 + j] = (int32_t)alias_draw(W->T.n_nodes, W->T.thr_n, W->T.alias_n, w[0], w[1], w[2]);
    }
}

int orc_sample_walk(int64_t n_nodes, int64_t n_arcs, const int32_t* src, const int32_t* dst,
                    const uint32_t* thr_e, const uint32_t* alias_e, const uint32_t* thr_n, const uint32_t* alias_n,
                    const double* cw, uint64_t seed, uint64_t t0, int64_t count, int K, int L, int Wn,
                    int reuse, int32_t* out) {
    if (L < 1 || Wn < 1 || Wn > L || reuse < 1) return -1;
    orc_walker W = {{n_nodes, n_arcs, src, dst, thr_e, alias_e, thr_n, alias_n}, cw, reuse};
    int32_t* nodes = (int32_t*)malloc(sizeof(int32_t) * (size_t)(L + 1));
    if (!nodes) return -2;
    int64_t cached = -1;
    for (int64_t i = 0; i < count; ++i)
        sample_walk_one(&W, seed, t0 + (uint64_t)i, K, L, Wn, nodes, &cached, out + i * (K + 2));
    free(nodes);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Initialisation: U[i][k] = ((w >> 8) - 2^23) * 2^-24 / dim, w = word       */
/* (k mod 4) of the draw at counter (i_lo, i_hi, k / 4, 1): uniform on       */
/* [-0.5/dim, 0.5/dim).  C = 0.                                              */
/* ------------------------------------------------------------------------ */
void orc_init_uniform(int64_t n, int dim, uint64_t seed, double* U) {
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < dim; ++k) {
            uint32_t w[4];
            draw_words(seed, 1, (uint64_t)i, (uint32_t)(k / 4), w);
            int32_t q = (int32_t)(w[k % 4] >> 8) - (1 << 23);
            U[i * dim + k] = ((double)q * (1.0 / 16777216.0)) / (double)dim;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Minibatch-synchronous LINE (Algorithm 1 with Eq. 2-4).                    */
/* ------------------------------------------------------------------------ */
static double sigmoid(double s) { return 1.0 / (1.0 + exp(-s)); }

static double dot(const double* a, const double* b, int dim) {
    double s = 0.0;
    for (int k = 0; k < dim; ++k) s += a[k] * b[k];
    return s;
}

/* eta_b = lr0 (schedule 0) or lr0 * max(1 - t0 / T, floor_frac) (schedule 1),
 * t0 the first global sample index of the batch. */
double orc_batch_lr(double lr0, int schedule, double floor_frac, uint64_t T, uint64_t t0) {
    if (schedule == 0) return lr0;
    double f = 1.0 - (double)t0 / (double)T;
    if (f < floor_frac) f = floor_frac;
    return lr0 * f;
}

/* Trains n_samples samples starting at global index sample_offset, in batches
 * of `batch` consecutive samples.  For each pair (x, y, label) of a sample:
 *   s = U_b[x] . Ctx_b[y],  g = eta_b (1 - sigma(s)) (label 1)
 *                             g = -eta_b alpha_neg sigma(s) (label 0),
 *   dU[x]   += g Ctx_b[y] - eta_b lambda U_b[x]
 *   dCtx[y] += g U_b[x]   - eta_b lambda Ctx_b[y]
 * where _b is the state at the start of the batch; after the batch X += dX.
 * order 2: Ctx = C (a separate table); order 1: Ctx = U (C is unused).
 * lr_total is T of the schedule (0 means sample_offset + n_samples). */
/* ------------------------------------------------------------------------ */
/* BF16 tables with stochastic rounding (a storage mode of the target; the   */
/* paper's tables are FP32).  A value written back is first the exact sum    */
/* X_b + dX rounded to FP32 (nearest), then rounded to BF16 stochastically:  */
/* 16 random bits r are added to the FP32 bit pattern below the BF16         */
/* mantissa and the low 16 bits are dropped; Inf and NaN pass unchanged.     */
/* Over the 2^16 equally likely r the expected BF16 value is the FP32 value  */
/* exactly.  The bits for the values 4k4 .. 4k4+3 of `row` of table `table`  */
/* (0: U, 1: C) written by the batch whose first sample is t0: with the      */
/* batch's salt s = SplitMix64 output function (Steele, Lea, Flood, OOPSLA   */
/* 2014) of seed ^ (t0 * 0x9E3779B97F4A7C15) (mod 2^64), the words           */
/*   w_j = fmix32(lo32(s) + (2 row + table) * 0x9E3779B1 + 2 k4 + j)         */
/* (mod 2^32, j = 0, 1; fmix32 is the 32-bit finaliser of Appleby's          */
/* MurmurHash3) form the 64 bits w_1 : w_0; value i of the four takes bits   */
/* [16 i, 16 i + 16).                                                        */
/* ------------------------------------------------------------------------ */
uint64_t orc_splitmix64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* MurmurHash3's 32-bit finaliser (fmix32). */
uint32_t orc_fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

uint64_t orc_sr_bits(uint64_t seed, uint32_t table, uint64_t row, uint64_t t0, uint32_t k4) {
    const uint64_t s = orc_splitmix64_mix(seed ^ (t0 * 0x9E3779B97F4A7C15ull));
    const uint32_t base = (uint32_t)s + (uint32_t)(2 * row + table) * 0x9E3779B1u + 2u * k4;
    const uint32_t w0 = orc_fmix32(base), w1 = orc_fmix32(base + 1u);
    return ((uint64_t)w1 << 32) | w0;
}

static uint32_t f32_bits(float x) {
    uint32_t b;
    memcpy(&b, &x, 4);
    return b;
}

static double bf16_bits_value(uint16_t h) {
    uint32_t b = (uint32_t)h << 16;
    float f;
    memcpy(&f, &b, 4);
    return (double)f;
}

/* BF16 bit pattern of FP32 x rounded stochastically with the 16 bits r16. */
uint16_t orc_bf16_sr_bits(float x, uint32_t r16) {
    uint32_t b = f32_bits(x);
    if ((b & 0x7F800000u) != 0x7F800000u) b += r16 & 0xFFFFu;
    return (uint16_t)(b >> 16);
}

/* BF16 bit pattern of FP32 x rounded to nearest, ties to even (NaN kept). */
uint16_t orc_bf16_rn_bits(float x) {
    uint32_t b = f32_bits(x);
    if ((b & 0x7F800000u) == 0x7F800000u) return (uint16_t)(b >> 16) | ((b & 0xFFFFu) ? 0x40u : 0u);
    uint32_t lsb = (b >> 16) & 1u;
    b += 0x7FFFu + lsb;
    return (uint16_t)(b >> 16);
}

/* Row v of a BF16 table after the batch starting at t0: X_b + dX, rounded. */
static void bf16_write_row(double* X, const double* dX, int64_t v, int dim, uint64_t seed, uint32_t table,
                           uint64_t t0) {
    for (int k = 0; k < dim; ++k) {
        float f = (float)(X[v * dim + k] + dX[v * dim + k]);
        uint64_t r = orc_sr_bits(seed, table, (uint64_t)v, t0, (uint32_t)(k / 4));
        uint32_t r16 = (uint32_t)(r >> (16 * (k % 4))) & 0xFFFFu;
        X[v * dim + k] = bf16_bits_value(orc_bf16_sr_bits(f, r16));
    }
}

static int train_minibatch(int64_t n_nodes, int64_t n_arcs, const int32_t* src, const int32_t* dst,
                           const uint32_t* thr_e, const uint32_t* alias_e, const uint32_t* thr_n,
                           const uint32_t* alias_n, int order, int dim, int K, double lr0, int schedule,
                           double lr_floor_frac, uint64_t lr_total, uint64_t n_samples, uint64_t seed, int64_t batch,
                           double lambda, double alpha_neg, uint64_t sample_offset, double* U, double* C,
                           const double* walk_cw, int walk_len, int window, int walk_reuse, int bf16) {
    if (batch <= 0 || dim <= 0 || K < 0 || (order != 1 && order != 2)) return -1;
    if (walk_cw && (walk_len < 1 || window < 1 || window > walk_len || walk_reuse < 1)) return -1;
    orc_tables T = {n_nodes, n_arcs, src, dst, thr_e, alias_e, thr_n, alias_n};
    orc_walker Wk = {T, walk_cw, walk_reuse};
    int32_t* wnodes = walk_cw ? (int32_t*)malloc(sizeof(int32_t) * (size_t)(walk_len + 1)) : NULL;
    int64_t wcached = -1;
    double* Ctx = order == 2 ? C : U;
    double* dU = (double*)calloc((size_t)n_nodes * (size_t)dim, sizeof(double));
    double* dC = order == 2 ? (double*)calloc((size_t)n_nodes * (size_t)dim, sizeof(double)) : dU;
    char* touchU = (char*)calloc((size_t)n_nodes, 1);
    char* touchC = order == 2 ? (char*)calloc((size_t)n_nodes, 1) : touchU;
    int32_t* rows = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * batch * (K + 2)));
    int32_t* rec = (int32_t*)malloc(sizeof(int32_t) * (size_t)(K + 2));
    if (!dU || !dC || !touchU || !touchC || !rows || !rec) return -2;
    uint64_t Ttot = lr_total ? lr_total : sample_offset + n_samples;
    uint64_t end = sample_offset + n_samples;
    for (uint64_t t0 = sample_offset; t0 < end; t0 += (uint64_t)batch) {
        uint64_t t1 = t0 + (uint64_t)batch < end ? t0 + (uint64_t)batch : end;
        double eta = orc_batch_lr(lr0, schedule, lr_floor_frac, Ttot, t0);
        int64_t nrows_u = 0, nrows_c = 0;
        int32_t* rows_u = rows;
        int32_t* rows_c = rows + batch * (K + 2);
        for (uint64_t t = t0; t < t1; ++t) {
            if (walk_cw) sample_walk_one(&Wk, seed, t, K, walk_len, window, wnodes, &wcached, rec);
            else sample_one(&T, seed, 0, t, K, rec);
            int32_t x = rec[0];
            for (int j = 0; j <= K; ++j) {
                int32_t y = rec[1 + j];
                double label = j == 0 ? 1.0 : 0.0;
                const double* ux = U + (int64_t)x * dim;
                const double* cy = Ctx + (int64_t)y * dim;
                double s = dot(ux, cy, dim);
                double g = j == 0 ? eta * (label - sigmoid(s)) : -eta * alpha_neg * sigmoid(s);
                double* dux = dU + (int64_t)x * dim;
                double* dcy = dC + (int64_t)y * dim;
                for (int k = 0; k < dim; ++k) {
                    dux[k] += g * cy[k] - eta * lambda * ux[k];
                    dcy[k] += g * ux[k] - eta * lambda * cy[k];
                }
                if (!touchU[x]) { touchU[x] = 1; rows_u[nrows_u++] = x; }
                if (!touchC[y]) {
                    touchC[y] = 1;
                    if (order == 2) rows_c[nrows_c++] = y;
                    else rows_u[nrows_u++] = y;
                }
            }
        }
        for (int64_t r = 0; r < nrows_u; ++r) {
            int64_t v = rows_u[r];
            if (bf16) bf16_write_row(U, dU, v, dim, seed, 0u, t0);
            else for (int k = 0; k < dim; ++k) U[v * dim + k] += dU[v * dim + k];
            for (int k = 0; k < dim; ++k) dU[v * dim + k] = 0.0;
            touchU[v] = 0;
        }
        for (int64_t r = 0; r < nrows_c; ++r) {
            int64_t v = rows_c[r];
            if (bf16) bf16_write_row(C, dC, v, dim, seed, 1u, t0);
            else for (int k = 0; k < dim; ++k) C[v * dim + k] += dC[v * dim + k];
            for (int k = 0; k < dim; ++k) dC[v * dim + k] = 0.0;
            touchC[v] = 0;
        }
    }
    free(rec);
    free(rows);
    free(wnodes);
    if (order == 2) { free(dC); free(touchC); }
    free(dU);
    free(touchU);
    return 0;
}

int orc_train(int64_t n_nodes, int64_t n_arcs, const int32_t* src, const int32_t* dst,
              const uint32_t* thr_e, const uint32_t* alias_e, const uint32_t* thr_n, const uint32_t* alias_n,
              int order, int dim, int K, double lr0, int schedule, double lr_floor_frac, uint64_t lr_total,
              uint64_t n_samples, uint64_t seed, int64_t batch, double lambda, double alpha_neg,
              uint64_t sample_offset, double* U, double* C, const double* walk_cw, int walk_len, int window,
              int walk_reuse) {
    return train_minibatch(n_nodes, n_arcs, src, dst, thr_e, alias_e, thr_n, alias_n, order, dim, K, lr0, schedule,
                           lr_floor_frac, lr_total, n_samples, seed, batch, lambda, alpha_neg, sample_offset, U, C,
                           walk_cw, walk_len, window, walk_reuse, 0);
}

/* The same batches on BF16 tables: U (and C) hold BF16 values (as doubles)
 * and every row written after a batch is rounded as described above. */
int orc_train_bf16(int64_t n_nodes, int64_t n_arcs, const int32_t* src, const int32_t* dst,
                   const uint32_t* thr_e, const uint32_t* alias_e, const uint32_t* thr_n, const uint32_t* alias_n,
                   int order, int dim, int K, double lr0, int schedule, double lr_floor_frac, uint64_t lr_total,
                   uint64_t n_samples, uint64_t seed, int64_t batch, double lambda, double alpha_neg,
                   uint64_t sample_offset, double* U, double* C, const double* walk_cw, int walk_len, int window,
                   int walk_reuse) {
    return train_minibatch(n_nodes, n_arcs, src, dst, thr_e, alias_e, thr_n, alias_n, order, dim, K, lr0, schedule,
                           lr_floor_frac, lr_total, n_samples, seed, batch, lambda, alpha_neg, sample_offset, U, C,
                           walk_cw, walk_len, window, walk_reuse, 1);
}

/* ------------------------------------------------------------------------ */
/* Per-pair immediate updates: the local path of Algorithm 1 with            */
/* LineUpdate, one pair after the other.  Samples t run in order, and the    */
/* pairs of a sample in the order (u, v), (u, n_1) .. (u, n_K).  One call:   */
/*   x = U[u], c = Ctx[y] (both read before either is written),              */
/*   s = x . c,  g = eta (1 - sigma(s)) (positive) or                        */
/*               g = -eta alpha_neg sigma(s) (negative),                     */
/*   U[u]  <- x + (g c - eta lambda x),                                      */
/*   Ctx[y] <- c + (g x - eta lambda c), written after U[u] (with order 1    */
/*   and y = u this value stays).                                            */
/* eta is the schedule's value at the first sample of t's block of `batch`   */
/* samples counted from sample_offset; pairs come from the arc sampler or,   */
/* with walk_cw, the walk sampler, as in orc_train.                          */
/* ------------------------------------------------------------------------ */
int orc_train_pairwise(int64_t n_nodes, int64_t n_arcs, const int32_t* src, const int32_t* dst,
                       const uint32_t* thr_e, const uint32_t* alias_e, const uint32_t* thr_n,
                       const uint32_t* alias_n, int order, int dim, int K, double lr0, int schedule,
                       double lr_floor_frac, uint64_t lr_total, uint64_t n_samples, uint64_t seed, int64_t batch,
                       double lambda, double alpha_neg, uint64_t sample_offset, double* U, double* C,
                       const double* walk_cw, int walk_len, int window, int walk_reuse) {
    if (batch <= 0 || dim <= 0 || K < 0 || (order != 1 && order != 2)) return -1;
    if (walk_cw && (walk_len < 1 || window < 1 || window > walk_len || walk_reuse < 1)) return -1;
    orc_tables T = {n_nodes, n_arcs, src, dst, thr_e, alias_e, thr_n, alias_n};
    orc_walker Wk = {T, walk_cw, walk_reuse};
    int32_t* wnodes = walk_cw ? (int32_t*)malloc(sizeof(int32_t) * (size_t)(walk_len + 1)) : NULL;
    int64_t wcached = -1;
    double* Ctx = order == 2 ? C : U;
    int32_t* rec = (int32_t*)malloc(sizeof(int32_t) * (size_t)(K + 2));
    double* x = (double*)malloc(sizeof(double) * (size_t)dim);
    double* c = (double*)malloc(sizeof(double) * (size_t)dim);
    if (!rec || !x || !c || (walk_cw && !wnodes)) return -2;
    uint64_t Ttot = lr_total ? lr_total : sample_offset + n_samples;
    uint64_t end = sample_offset + n_samples;
    for (uint64_t t = sample_offset; t < end; ++t) {
        uint64_t t0 = sample_offset + (t - sample_offset) / (uint64_t)batch * (uint64_t)batch;
        double eta = orc_batch_lr(lr0, schedule, lr_floor_frac, Ttot, t0);
        if (walk_cw) sample_walk_one(&Wk, seed, t, K, walk_len, window, wnodes, &wcached, rec);
        else sample_one(&T, seed, 0, t, K, rec);
        double* urow = U + (int64_t)rec[0] * dim;
        for (int j = 0; j <= K; ++j) {
            double* crow = Ctx + (int64_t)rec[1 + j] * dim;
            for (int k = 0; k < dim; ++k) { x[k] = urow[k]; c[k] = crow[k]; }
            double s = dot(x, c, dim);
            double g = j == 0 ? eta * (1.0 - sigmoid(s)) : -eta * alpha_neg * sigmoid(s);
            for (int k = 0; k < dim; ++k) urow[k] = x[k] + (g * c[k] - eta * lambda * x[k]);
            for (int k = 0; k < dim; ++k) crow[k] = c[k] + (g * x[k] - eta * lambda * c[k]);
        }
    }
    free(c);
    free(x);
    free(rec);
    free(wnodes);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Multi-threaded CPU Hogwild in FP32 - context for the benchmark, not a     */
/* reference: the per-pair updates of orc_train_pairwise on FP32 tables,     */
/* with `threads` POSIX threads; thread i takes samples i, i + threads, ...  */
/* and reads and writes the shared rows without locks, as multi-threaded     */
/* CPU LINE does.  With one thread it is the sequential per-pair run in      */
/* FP32.                                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    orc_tables T;
    int order, dim, K, schedule;
    double lr0, floor_frac;
    uint64_t Ttot, n_samples, seed, offset;
    int64_t batch;
    float lambda, alpha_neg;
    float *U, *C;
    int tid, threads, status;
} orc_hog_job;

static void* orc_hog_worker(void* arg) {
    orc_hog_job* j = (orc_hog_job*)arg;
    const int dim = j->dim;
    int32_t* rec = (int32_t*)malloc(sizeof(int32_t) * (size_t)(j->K + 2));
    float* x = (float*)malloc(sizeof(float) * (size_t)dim);
    float* c = (float*)malloc(sizeof(float) * (size_t)dim);
    if (!rec || !x || !c) {
        j->status = -2;
        free(rec); free(x); free(c);
        return NULL;
    }
    float* Ctx = j->order == 2 ? j->C : j->U;
    for (uint64_t i = (uint64_t)j->tid; i < j->n_samples; i += (uint64_t)j->threads) {
        const uint64_t t = j->offset + i;
        const uint64_t t0 = j->offset + i / (uint64_t)j->batch * (uint64_t)j->batch;
        const float eta = (float)orc_batch_lr(j->lr0, j->schedule, j->floor_frac, j->Ttot, t0);
        sample_one(&j->T, j->seed, 0, t, j->K, rec);
        float* urow = j->U + (int64_t)rec[0] * dim;
        for (int k = 0; k <= j->K; ++k) {
            float* crow = Ctx + (int64_t)rec[1 + k] * dim;
            float sdot = 0.0f;
            for (int e = 0; e < dim; ++e) {
                x[e] = urow[e];
                c[e] = crow[e];
                sdot += x[e] * c[e];
            }
            const float sig = 1.0f / (1.0f + expf(-sdot));
            const float g = k == 0 ? eta * (1.0f - sig) : -eta * j->alpha_neg * sig;
            for (int e = 0; e < dim; ++e) urow[e] = x[e] + (g * c[e] - eta * j->lambda * x[e]);
            for (int e = 0; e < dim; ++e) crow[e] = c[e] + (g * x[e] - eta * j->lambda * c[e]);
        }
    }
    free(rec); free(x); free(c);
    return NULL;
}

int orc_train_hogwild_mt(int64_t n_nodes, int64_t n_arcs, const int32_t* src, const int32_t* dst,
                         const uint32_t* thr_e, const uint32_t* alias_e, const uint32_t* thr_n,
                         const uint32_t* alias_n, int order, int dim, int K, double lr0, int schedule,
                         double lr_floor_frac, uint64_t lr_total, uint64_t n_samples, uint64_t seed, int64_t batch,
                         double lambda, double alpha_neg, uint64_t sample_offset, float* U, float* C, int threads) {
    if (batch <= 0 || dim <= 0 || K < 0 || (order != 1 && order != 2) || threads < 1 || threads > 1024) return -1;
    orc_hog_job* jobs = (orc_hog_job*)calloc((size_t)threads, sizeof(orc_hog_job));
    pthread_t* th = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -2; }
    int rc = 0, started = 0;
    for (int i = 0; i < threads; ++i) {
        orc_hog_job* j = &jobs[i];
        j->T = (orc_tables){n_nodes, n_arcs, src, dst, thr_e, alias_e, thr_n, alias_n};
        j->order = order; j->dim = dim; j->K = K; j->schedule = schedule;
        j->lr0 = lr0; j->floor_frac = lr_floor_frac;
        j->Ttot = lr_total ? lr_total : sample_offset + n_samples;
        j->n_samples = n_samples; j->seed = seed; j->offset = sample_offset; j->batch = batch;
        j->lambda = (float)lambda; j->alpha_neg = (float)alpha_neg;
        j->U = U; j->C = C; j->tid = i; j->threads = threads;
        if (pthread_create(&th[i], NULL, orc_hog_worker, j) != 0) { rc = -3; break; }
        ++started;
    }
    for (int i = 0; i < started; ++i) {
        pthread_join(th[i], NULL);
        if (jobs[i].status) rc = jobs[i].status;
    }
    free(jobs);
    free(th);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Negative-sampling LINE loss over m fixed samples (draw domain 3):         */
/*   L = - sum_t [ log sigma(s+) + sum_j log sigma(-s-_j) ]                  */
/* with s = U[u] . Ctx[y] (Ctx = C for order 2, U for order 1).              */
/* ------------------------------------------------------------------------ */
static double log_sigmoid(double s) {
    /* log sigma(s) = -(max(-s, 0) + log1p(exp(-|s|))) */
    double a = s < 0.0 ? -s : 0.0;
    return -(a + log1p(exp(-fabs(s))));
}

double orc_eval_loss(int64_t n_nodes, int64_t n_arcs, const int32_t* src, const int32_t* dst,
                     const uint32_t* thr_e, const uint32_t* alias_e, const uint32_t* thr_n, const uint32_t* alias_n,
                     int order, int dim, int K, uint64_t seed, int64_t m, const double* U, const double* C) {
    orc_tables T = {n_nodes, n_arcs, src, dst, thr_e, alias_e, thr_n, alias_n};
    const double* Ctx = order == 2 ? C : U;
    int32_t* rec = (int32_t*)malloc(sizeof(int32_t) * (size_t)(K + 2));
    double L = 0.0;
    for (int64_t t = 0; t < m; ++t) {
        sample_one(&T, seed, 3, (uint64_t)t, K, rec);
        const double* ux = U + (int64_t)rec[0] * dim;
        for (int j = 0; j <= K; ++j) {
            double s = dot(ux, Ctx + (int64_t)rec[1 + j] * dim, dim);
            L -= j == 0 ? log_sigmoid(s) : log_sigmoid(-s);
        }
    }
    free(rec);
    return L;
}
