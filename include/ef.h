/*
 * ef.h -- C ABI of libef.so: the Expected Force (EF_2) of every node of an
 * undirected simple graph, computed by hand-written sm_103a CUDA kernels.
 *
 * Method (paper "Scaling Expected Force", Sections 3.3 and 4): a 2-hop
 * transmission cluster is a tree with two edges; its out-degree d is the
 * number of edges leaving it.  Algorithm 1 enumerates every cluster once as
 * a triple (i, v, j) of a middle node v and two of its neighbours i < j,
 * with d = D_v + D_i + D_j - 4, minus 2 more when i and j are adjacent, and
 * credits d once to i, once to j and twice to v.  EF(v) is the entropy of
 * the normalised degrees of the clusters credited to v (Eq. 1), which equals
 *     EF(v) = ln S_v - T_v / S_v,  S_v = sum of credited d,
 *                                  T_v = sum of credited d ln d.
 * A node whose credited degrees sum to 0 (no clusters, or only clusters of
 * degree 0) is degenerate: EF = 0 and its flag is 1.
 *
 * Graph format (all entry points): symmetric CSR, int32 indices.
 *   row_ptr[n+1], row_ptr[0] = 0, row_ptr[n] = m, non-decreasing;
 *   col_idx[m]: each undirected edge stored in both rows (m = nnz = 2|E|),
 *   every row strictly ascending, no self-loops, entries in [0, n).
 *   m must be < 2^31.
 *
 * Memory: the caller owns every input and output buffer.  Pointers are
 * device pointers unless ef_options.host_io = 1.  A context owns its device
 * scratch, grows it on demand and frees it in ef_ctx_destroy.  Work is
 * issued on the context's stream; ef_compute_ex returns after the stream has
 * finished unless ef_options.async = 1 (see there).
 *
 * Errors: every entry point returns an int status (no exceptions cross the
 * ABI).  ef_last_error(ctx) gives a one-line message for the last failure.
 */
#ifndef EF_H
#define EF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum ef_status {
    EF_OK = 0,
    EF_ERR_ARG = 1,         /* null pointer, negative size, m >= 2^31, bad option */
    EF_ERR_GRAPH = 2,       /* not a symmetric simple sorted CSR (checked on device) */
    EF_ERR_OOM = 3,         /* device or pinned allocation failed */
    EF_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    EF_ERR_TIMEOUT = 5,     /* reserved: no call returns it (no kernel of
                               this library waits on a flag or on another
                               device, so there is no watchdog) */
    EF_ERR_MODEL = 6,       /* surrogate model malformed or mismatched */
    EF_ERR_UNSUPPORTED = 7  /* option combination not provided, or a node
                               of degree above EF_MAX_DEGREE */
};

enum ef_precision {
    EF_PREC_FP64 = 0,  /* d ln d computed in FP64 (a table held as FP32
                          pairs, within 2^-48); row sums in FP32-pair
                          chunks of at most 32 terms (below 3.6e-12
                          relative each), everything else in FP64, ln S
                          and T/S by a table-based logarithm and a refined
                          reciprocal (about 1e-14 relative).  EF within
                          1e-9 relative of the exact value */
    EF_PREC_FP32C = 1  /* d ln d in FP32 (hardware log2) with compensated
                          (Kahan) FP32 sums per thread; the credits a node
                          receives from its neighbours are summed in FP64;
                          ln S - T/S in FP32 (FP64 above degree 1000).
                          EF within 2e-5 absolute of the exact value */
};

/* Largest maximum degree a validated call accepts: the exact integer sums S_v
 * (and their closed forms' products) stay below 2^63 up to it (S_v is at
 * most 6 maxdeg^3).  A validated graph with a node of larger degree gives
 * EF_ERR_UNSUPPORTED; with trust_input the caller guarantees it. */
#define EF_MAX_DEGREE (1 << 20)

typedef struct ef_ctx ef_ctx;

typedef struct {
    const int32_t *row_ptr;   /* n+1 entries */
    const int32_t *col_idx;   /* m entries */
} ef_csr;

typedef struct {
    int32_t precision;     /* enum ef_precision; default EF_PREC_FP64 */
    int32_t trust_input;   /* 1: skip CSR validation (and its host sync) */
    int32_t host_io;       /* 1: graph and outputs are host pointers; the
                              library copies them in and out */
    int32_t async;         /* 1: return once the work is queued on the
                              context stream (with validation, after its
                              readback midway); results, in device or host
                              buffers, are valid after ef_sync, and host
                              buffers must stay valid and unchanged until
                              then.  Two contexts on two streams then overlap
                              one call's copies with another's kernels. */
    int32_t profile;       /* 1: time each pass with CUDA events on the
                              context stream (read with ef_get_stats) */
    int32_t wedge_mode;    /* 0: automatic (degree-class kernels for middle
                              nodes of degree > 32); 1: the direct pairwise
                              wedge kernel for every middle node of degree
                              > 32 (reference kernel for benchmarking); other
                              values: EF_ERR_UNSUPPORTED */
    int32_t graph;         /* 1: run the passes that need no host decision as
                              one CUDA graph, captured on the first call and
                              replayed while pointers, sizes, options and
                              tuning stay the same (ignored with profile) */
    int32_t device_check;  /* 1: validate on the device with no readback in
                              the middle of the call (ignored with
                              trust_input).  The kernels after the
                              validation do nothing when it failed, so the
                              whole call -- validation included -- is one
                              CUDA graph with graph = 1.  A synchronous call
                              reads the validation result once at its end and
                              returns EF_ERR_GRAPH or EF_ERR_UNSUPPORTED as
                              without device_check; with async the next
                              ef_sync returns that error (any failed call
                              since the previous ef_sync).  On an error the
                              device outputs are not written (with host_io
                              the host buffers' contents are undefined).  The
                              layout of the oriented lists is then chosen
                              without the readback (ef_tuning.layout), and
                              the f table is sized for min(n - 1, m,
                              EF_MAX_DEGREE).
                              Read by ef_compute_ex and ef_compute_batched;
                              the other calls ignore it. */
} ef_options;

/* Optional per-node outputs (any may be NULL); length n each. */
typedef struct {
    double  *ef;          /* EF(v) */
    int64_t *n_clusters;  /* N_v: number of credited clusters (weights 2/1/1) */
    int64_t *s;           /* S_v: sum of credited cluster degrees (exact) */
    double  *t;           /* T_v: sum of credited d ln d */
    int64_t *triangles;   /* t_v: triangles through v */
    uint8_t *flag;        /* 1: degenerate (S_v = 0), EF = 0 */
} ef_outputs;

/* Per-pass timings in milliseconds, summed over profiled calls (CUDA events
 * on the context stream between the passes). */
typedef struct {
    int64_t calls;
    double prep_ms;        /* validation, degrees, neighbour sums */
    double orient_ms;      /* f table, degree orientation (scan + oriented
                              CSR + out-list hash tables) and omega */
    double wedge_small_ms; /* middle nodes of degree <= 32 */
    double wedge_big_ms;   /* middle nodes of degree > 32 */
    double tri_hash_ms;    /* always 0: the orientation builds the hash
                              tables of the long out-lists (orient_ms) */
    double tri_pairs_ms;   /* triangle pair tests and corrections (one kernel) */
    double finalize_ms;    /* per-node sums, S, N, EF */
    double total_ms;
    int64_t kernels;       /* kernels launched by profiled calls */
    int64_t graph_replays; /* calls served by replaying a cached CUDA graph */
} ef_stats;

/* Launch parameters (every choice gives the same results; see ef_autotune). */
typedef struct {
    int32_t row_thread_max; /* row passes: rows of degree <= this are walked by
                               one thread, longer ones by a warp (1..32; 32) */
    int32_t hub_min;        /* rows and middle nodes of degree >= this take a
                               whole CTA (33..513; 513) */
    int32_t tri_variant;    /* pair-test kernel: 0 two candidates per lane
                               step, 1 four (0) */
    int32_t grid_per_sm;    /* blocks per SM of the grid-stride row passes
                               (1..256; 64) */
    int32_t layout;         /* order of the oriented out-lists: 1 node order
                               (keeps a graph's own locality), 2 by degree
                               class (lists of similar degree share cache
                               lines), 0 automatic: degree classes when the
                               nodes of degree > 32 span more than half of
                               the ids, else node order; with trust_input
                               (nothing read back) degree classes for one
                               graph and node order for a batch (0) */
} ef_tuning;

/* Create a context on CUDA device `device` issuing work on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  0 on success. */
int ef_ctx_create(int device, void *stream, ef_ctx **out);
/* Cap the device memory the context may hold for its working buffers
 * (scratch, f tables, staging copies, batch offsets, learned-path and SIR
 * buffers; models are separate), in bytes; 0 = no cap (the default).  A call
 * that would need more returns EF_ERR_OOM with a message naming both sizes,
 * before it frees or allocates anything, and leaves the context usable (a
 * later call with a higher cap, or on a smaller graph, runs normally).
 * Lowering the cap frees nothing already held. */
int ef_ctx_set_memory_limit(ef_ctx *ctx, uint64_t bytes);
/* Free the context and its scratch.  Safe on NULL. */
int ef_ctx_destroy(ef_ctx *ctx);
/* Message of the last failure on this context ("" if none); ctx may be
 * NULL for failures of ef_compute and ef_ctx_create. */
const char *ef_last_error(const ef_ctx *ctx);
/* Wait for all work issued on the context's stream.  Returns EF_ERR_GRAPH
 * or EF_ERR_UNSUPPORTED when an asynchronous call with device_check since
 * the previous ef_sync failed its validation (the message names the bits of
 * all of them), else EF_OK or EF_ERR_CUDA. */
int ef_sync(ef_ctx *ctx);
/* Read (and with reset != 0, clear) the accumulated pass timings. */
int ef_get_stats(ef_ctx *ctx, ef_stats *out, int reset);

/*
 * EF of every node (Algorithm 1, Eq. 1).  Device pointers; FP64 path;
 * input validated; synchronous on the current device's legacy default
 * stream, with a library-owned context per device.
 *   g: CSR (device), n: nodes, m: nnz, out_ef: double[n] (device).
 * Returns EF_OK or an ef_status code.
 */
int ef_compute(const ef_csr *g, int32_t n, int64_t m, double *out_ef);

/*
 * Full-control form of ef_compute: options (NULL = defaults) and optional
 * per-node outputs N, S, T, t, flag besides EF.
 */
int ef_compute_ex(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m,
                  const ef_options *opt, ef_outputs *out);

/*
 * Batched EF (many graphs in one call).  The batch is one CSR over the
 * disjoint union of its graphs with global node ids: graph k owns nodes
 * [graph_off[k], graph_off[k+1]) and every entry of those rows lies in the
 * same range.  EF of a node depends only on nodes within two hops of it
 * (Algorithm 1 credits a node only for clusters that contain it), so EF over
 * the union equals EF of each graph computed alone.
 *   g: union CSR (device unless host_io), m: its nnz (< 2^31);
 *   graph_off: int64[num_graphs+1], HOST memory, graph_off[0] = 0,
 *   non-decreasing, n = graph_off[num_graphs] < 2^31;
 *   out: per-node outputs over the union (length n).
 * Validation (unless trust_input) is ef_compute_ex's plus the check that no
 * entry leaves its graph (EF_ERR_GRAPH "edge-between-graphs").  With
 * opt->graph = 1 the passes run as one replayed CUDA graph (with
 * trust_input, the whole call is one graph launch).
 */
int ef_compute_batched(ef_ctx *ctx, const ef_csr *g, int64_t m,
                       const int64_t *graph_off, int32_t num_graphs,
                       const ef_options *opt, ef_outputs *out);

/* Read or set the context's launch parameters (t = NULL restores the
 * defaults; out-of-range values give EF_ERR_ARG and change nothing). */
int ef_get_tuning(const ef_ctx *ctx, ef_tuning *out);
int ef_set_tuning(ef_ctx *ctx, const ef_tuning *t);

/*
 * Autotuner: validates the graph once (unless trust_input), then times
 * candidate launch parameters on it (coordinate descent over the five
 * ef_tuning fields, two sweeps; each candidate one warm-up and `reps` timed
 * runs as a replayed CUDA graph, CUDA events on the context stream), keeps
 * the fastest on the context and returns it in *best.  A batch is tuned by
 * passing its union CSR.  Device pointers only.
 */
int ef_autotune(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m,
                const ef_options *opt, int32_t reps, ef_tuning *best);

/*
 * Exact EF of chosen nodes only (vertex-centric form of Algorithm 1: every
 * cluster containing a chosen node, with its 2/1/1 credits).
 *   g: CSR (device); nodes: int32[k] device node ids (duplicates allowed;
 *   an id outside [0, n) gives EF_ERR_ARG); out: device arrays of length k
 *   (out->ef[i] belongs to nodes[i]; any member may be NULL).
 * Validation and precision as ef_compute_ex (host_io and async are not
 * accepted: EF_ERR_ARG).
 */
int ef_compute_nodes(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m,
                     const int32_t *nodes, int32_t k, const ef_options *opt,
                     ef_outputs *out);

/* ------------------------------------------------------------------------
 * Sharded computation (Eq. 1 split over workers).  Every term of T_v comes
 * from one cluster, counted at its middle node, and every triangle
 * correction from one triangle, counted at its lowest-ranked node in the
 * (degree, id) order.  So R workers that each hold the whole CSR can split
 * Algorithm 1's cluster loop: shard r owns the nodes [lo, hi), lo the first
 * row that starts at or after adjacency entry r m / R, takes the clusters
 * and triangles counted at its nodes, and writes per-node partials, plus the
 * closed-form sums N_v and S_v + 8 t_v of its own nodes.  The element-wise
 * sum of the R partials (the one exchange: an all-reduce of 40 bytes per
 * node) gives ef_finalize_partials, an element-wise pass with no graph
 * input, the same N, S and triangle counts as ef_compute_ex, and EF within
 * its precision's bound (T's FP64 sum depends on the order of additions).
 * ---------------------------------------------------------------------- */
typedef struct {
    double  *t;          /* this shard's part of T_v at open degrees (its
                            clusters counted without triangle corrections) */
    int64_t *q;          /* triangle corrections to T_v, units of
                            2^-frac_bits */
    int64_t *triangles;  /* triangles through v that this shard listed */
    int64_t *n_clusters; /* N_v for v in the shard's range, else 0 */
    int64_t *s_open;     /* S_v + 8 t_v for v in the shard's range, else 0 */
} ef_partials;

/*
 * Partials of shard `shard` of `num_shards` (0 <= shard < num_shards).
 *   g: CSR (device); out: five device arrays of length n, all required;
 *   they are overwritten, not accumulated into;
 *   frac_bits (host, may be NULL): the fixed-point scale of q, the same for
 *   every shard of one graph; range (host int32[2], may be NULL): the
 *   shard's nodes [range[0], range[1]) (empty when R exceeds the rows).
 * Validation and precision as ef_compute_ex (every shard validates the
 * whole graph unless trust_input); host_io and async give EF_ERR_ARG.
 * Shards may run on different devices or one after another.
 */
int ef_compute_shard(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m,
                     int32_t shard, int32_t num_shards, const ef_options *opt,
                     ef_partials *out, int32_t *frac_bits, int32_t *range);

/*
 * EF from partials summed over all shards of one graph: five device arrays
 * of length n (q in units of 2^-frac_bits, 0..52, as ef_compute_shard
 * reported).  Writes any requested member of *out (device arrays of length
 * n) as ef_compute_ex would; reads no graph.  Only precision is read from
 * *opt; host_io and async give EF_ERR_ARG.
 */
int ef_finalize_partials(ef_ctx *ctx, int32_t n, const ef_partials *sum,
                         int32_t frac_bits, const ef_options *opt,
                         ef_outputs *out);

/* ------------------------------------------------------------------------
 * SIR epidemic simulation (Section 3.1's model, Section 3.2's measurements),
 * for checking how EF predicts a node's role in an epidemic.  Discrete,
 * synchronous time steps t = 0, 1, ...:
 *   - every node u infected at the start of step t tries once each
 *     neighbour x that is susceptible then; the try succeeds when
 *     R(sim, t, u, x) < floor(beta 2^32); x is infected at the end of the
 *     step if any try succeeded, and its infector (parent) is the smallest
 *     such u;
 *   - u recovers at the end of step t when R(sim, t, u, 2^32 - 1) <
 *     floor(gamma 2^32); immune nodes are never infected;
 *   - a simulation ends at the first t with no infected node (its length).
 * R is Philox4x32-10 (Salmon et al., SC 2011): counter (sim, t, u, x), key
 * = seed, first output word, with sim = sim_base + the simulation's index.
 * So a simulation's course depends on (seed, sim) only, and runs split
 * across calls or devices reproduce one long run.
 * Section 3.1 calibrates gamma = 1/3 and beta = 1.3 / (3 <k>).
 * ---------------------------------------------------------------------- */
typedef struct {
    double beta;            /* infection probability per try, [0, 1] */
    double gamma;           /* recovery probability per step, [0, 1] */
    uint64_t seed;          /* Philox key */
    int64_t sim_base;       /* id of simulation 0 of this call */
    int32_t max_steps;      /* >= 1; simulations still active then stop
                               there (length = max_steps, truncated = 1) */
    int32_t depth;          /* spreading-power orders 1..depth (0..4) */
    int32_t spread_min_size;/* only simulations whose final size is at
                               least this add to spread and spread_sims
                               (e.g. 25% of n: global outbreaks only) */
    int32_t reserved;
} ef_sir_params;

/* Outputs (device arrays; any may be NULL).  B = number of simulations. */
typedef struct {
    int32_t *final_size;    /* [B] nodes ever infected, index case included */
    int32_t *length;        /* [B] steps until no node is infected */
    int32_t *peak_infected; /* [B] most nodes infected at the start of a step */
    int32_t *peak_step;     /* [B] first step with that many */
    uint8_t *truncated;     /* [B] 1: still active after max_steps */
    int32_t *parent;        /* [B][n] infection tree: -1 never infected, the
                               index case is its own parent */
    int64_t *spread;        /* [depth][n] sum over the selected simulations
                               of the spreading power of order k: the nodes
                               of v's infection subtree within k generations
                               below v (v not counted) */
    int64_t *spread_sims;   /* [n] selected simulations in which v was
                               infected */
} ef_sir_outputs;

/*
 * Run num_sims simulations on graph g (device CSR, validated as in
 * ef_compute_ex unless opt->trust_input).
 *   index_cases: int32[num_sims] (device) start nodes;
 *   immune: uint8[num_immune_sets][n] (device, 1 = immune) or NULL, and
 *   immune_set: int32[num_sims] (device) the set of each simulation (-1:
 *   none) or NULL.
 * An index case outside [0, n) or immune, or a set index >= num_immune_sets,
 * gives EF_ERR_ARG before any step runs.  Simulations run in batches of up
 * to 1024 (one bit per simulation per node, node-major); device memory is
 * about 8 bytes per (simulation, node) pair of a batch.  host_io and async
 * give EF_ERR_ARG.
 */
int ef_sir_run(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m,
               const int32_t *index_cases, int32_t num_sims,
               const uint8_t *immune, int32_t num_immune_sets,
               const int32_t *immune_set, const ef_sir_params *params,
               const ef_options *opt, ef_sir_outputs *out);

/* ------------------------------------------------------------------------
 * Learned ranking path.  A regression network 16-64-64-1 (ReLU, BF16
 * tensor-core products with FP32 accumulation) maps 16 cheap per-node
 * features to a predicted EF.  It is trained on exact EF produced by this
 * library, ranks all nodes of a graph, and exact EF is then recomputed on
 * the best-ranked candidates and on a random audit sample.
 *
 * Features (row-major float32 [n][16], natural logarithms):
 *   0 ln(1+D)  1 ln(1+sigma1)  2 ln(1+sigma2)  3 ln(1+omega)
 *   4 ln(1+mean neighbour degree)  5 ln(1+its standard deviation)
 *   6 ln(1+min neighbour degree)   7 ln(1+max neighbour degree)
 *   8 ln(1+N)   9 ln(1+S_open)   10 = 9 - 8   11 ln(1+t)
 *   12 clustering t / C(D,2)   13 ln(1+S)   14 = 2 - 1   15 = 3 - 1
 * with sigma1, sigma2 the sums of neighbour degrees and of their squares,
 * omega the sum of the neighbours' sigma1, N the credited cluster count,
 * S_open the credited degree sum at open degrees, t the triangles and
 * S = S_open - 8t.  Feature mode 0 takes t = 0 (no triangle pass);
 * mode 1 runs the triangle pass.
 * ---------------------------------------------------------------------- */
typedef struct ef_model ef_model;

#define EF_MODEL_PARAMS 5313   /* W1[16][64], b1[64], W2[64][64], b2[64], w3[64], b3 */
#define EF_MODEL_FLOATS (EF_MODEL_PARAMS + 32)   /* followed by mean[16], std[16] */

/* Features of every node into x (device float32 [n*16]). */
int ef_features(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m,
                int32_t mode, const ef_options *opt, float *x);

/* A model on the context's device: weights uniform in
 * +-1/sqrt(fan in) from a counter-based generator (splitmix64 of seed),
 * zero biases, standardisation unset (fitted from the first training data). */
int ef_model_create(ef_ctx *ctx, uint64_t seed, int32_t feature_mode, ef_model **out);
int ef_model_destroy(ef_model *model);
/* Copy all EF_MODEL_FLOATS floats out of / into host memory (set marks the
 * standardisation as fitted). */
int ef_model_get(const ef_model *model, float *host);
int ef_model_set(ef_model *model, const float *host);
int ef_model_feature_mode(const ef_model *model);
/* Binary file: 8-byte magic "EFMLP001", int32 feature mode, int32 fitted,
 * EF_MODEL_FLOATS little-endian float32. */
int ef_model_save(const ef_model *model, const char *path);
int ef_model_load(ef_ctx *ctx, const char *path, ef_model **out);

/* Predictions for n feature rows (device x float32 [n*16], out float32 [n]). */
int ef_mlp_forward(ef_ctx *ctx, const ef_model *model, const float *x, int32_t n, float *out);
/* Mean-squared-error loss over all n rows and its gradient with respect to
 * the EF_MODEL_PARAMS parameters (device x, y; host loss and grad). */
int ef_mlp_grad(ef_ctx *ctx, ef_model *model, const float *x, const float *y, int32_t n,
                float *loss, float *grad);

typedef struct {
    int32_t steps;      /* Adam steps */
    int32_t batch;      /* rows per step, sampled uniformly with replacement
                           by a counter-based generator */
    float lr;           /* Adam step size (beta1 0.9, beta2 0.999, eps 1e-8) */
    int32_t pad;
    uint64_t seed;
} ef_train_options;

typedef struct {
    float first_loss, last_loss;   /* batch losses of the first and last step */
    double ms;                     /* device time of the whole training */
} ef_train_stats;

/* Train on n rows (device x float32 [n*16], y float32 [n] = exact EF).
 * The steps after the first replay one captured CUDA graph. */
int ef_surrogate_train(ef_ctx *ctx, ef_model *model, const float *x, const float *y, int32_t n,
                       const ef_train_options *opt, ef_train_stats *stats);

typedef struct {
    int32_t n_candidates;   /* nodes whose exact EF was recomputed as candidates */
    int32_t n_audit;        /* audit sample size */
    int32_t n_top;          /* size of the reported top set */
    int32_t pad;
    double spearman_audit;  /* Spearman rho of prediction vs exact EF on the audit sample */
    double max_abs_err_audit;
    double features_ms, infer_ms, select_ms, exact_ms, total_ms;
    double exact_tri_ms;    /* of exact_ms: the triangle pass */
    double exact_wedge_ms;  /* of exact_ms: marking, bins and the wedge pass */
} ef_rank_stats;

/*
 * Rank the nodes of g with the model:
 * - features, then predictions of every node;
 * - the ceil(cand_frac n) best-predicted nodes are the candidates;
 * - an audit sample takes each node with probability audit_frac (splitmix64
 *   of seed and node id);
 * - exact EF (ef_compute_nodes) of candidates and audit nodes;
 * - out_idx / out_ef (device, capacity ceil(top_frac n)) receive the
 *   ceil(top_frac n) candidates of largest exact EF, in node-id order.
 * The plain exact pass stays the reference: recall against it is
 * measured by the caller.  out_score (device float32 [n], may be NULL)
 * receives every prediction.  Requires 0 < top_frac <= cand_frac <= 1.
 */
int ef_surrogate_rank(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m, const ef_model *model,
                      float top_frac, float cand_frac, float audit_frac, uint64_t seed,
                      const ef_options *opt, int32_t *out_idx, double *out_ef, float *out_score,
                      ef_rank_stats *stats);

/*
 * ef_compute_static: EF of every node with no memory allocation at all.
 * The paper has no counterpart; this is for callers that cannot allocate
 * device memory when they need EF (code inside a memory pool that owns the
 * device, hosts that forbid cudaMalloc/cudaFree because they synchronise the
 * device, real-time loops that must not touch an allocator).
 *   g: CSR (device pointers), n, m as above; precision: enum ef_precision;
 *   out_ef: double[n] (device); stream: a cudaStream_t (NULL = legacy
 *   default stream) on the current device.  Synchronous: returns after the
 *   stream has finished this call's work.  Input is validated.
 * Scratch lives in a fixed 32 MiB device array inside the library, held by
 * every GPU that loads it until the process exits.  Graphs whose scratch
 * would exceed it (about 172 n + 44 m + 48 min(n, m) bytes) are rejected with
 * EF_ERR_ARG and a message naming the limit; nothing runs on the GPU then.
 * The first call on a device looks up the array's address (make it before
 * any stream capture).  Under CUDA's lazy module loading that first call is
 * also when the device's 32 MiB are reserved, so make it before a memory pool
 * takes the device; a call with n = 0 does only this set-up (a failure to
 * reserve gives EF_ERR_OOM).  The address is cached until the process exits:
 * it is not valid across a cudaDeviceReset of the device.  All calls share
 * the array, which keeps the previous call's contents (each call clears what
 * must start at zero): calls that overlap on the GPU race and must be
 * serialised by the caller.  Errors: ef_last_error(NULL).
 */
int ef_compute_static(const ef_csr *g, int32_t n, int64_t m, int32_t precision,
                      double *out_ef, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* EF_H */
