// C ABI of libef (declared in include/ef.h): contexts, scratch management,
// the orchestration of the passes, batched input, CUDA-graph replay and the
// autotuner.
//
// Pass order (one graph or one batch, all on the context stream):
//   part A   one memset of the per-node accumulators and the counters;
//            degrees + row_ptr checks + wedge bins; per-row checks,
//            sigma1/sigma2, out-degrees, symmetry fingerprints; (batched)
//            the check that no entry leaves its graph
//   host     one small readback: validation word and max degree
//            (skipped with trust_input)
//   part B   f table (f(d) = d ln d and the triangle corrections, d < 3 maxdeg + 1);
//            orientation (oriented CSR + omega); wedge pass (small, then mid +
//            hub middle nodes); hash tables and pair tests; finalize (per node)
//   host     final readback of the validation word (asymmetric input is
//            only detected by the finalize pass)
// The wedge pass and the orientation + triangle passes write disjoint
// accumulators and could run on two streams; measured on the 4M-node
// power-law graph, the concurrent form was slower (the triangle pass more
// than doubles under contention), so they run in sequence.
//
// CUDA graphs (ef_options.graph): the part that needs no host decision --
// part B, or parts A and B together under trust_input -- is captured once on
// a private stream and replayed into the context stream while the pointers,
// sizes, options and tuning stay the same (one cached graph per context).
#include "ef_internal.cuh"

#include <mutex>
#include <new>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

namespace {

// What a captured graph depends on: replayed only when every byte matches
// (the layout has no padding; keys are zero-filled before use).
struct GraphKey {
    const void *rp, *ci, *goff_dev, *scratch, *ftab;
    const void *outs[6];
    int64_t m, fcap;
    int32_t n, G, precision, wedge_mode, trust, pad;
    ef::Tune tune;
    int32_t pad2;
    bool operator==(const GraphKey &o) const { return memcmp(this, &o, sizeof *this) == 0; }
};
static_assert(sizeof(GraphKey) == 11 * 8 + 2 * 8 + 6 * 4 + sizeof(ef::Tune) + 4, "GraphKey has padding");

}  // namespace

struct ef_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;   // private stream for graph capture
    int num_sms = 0;
    char err[512] = {0};
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    double *ftab = nullptr;
    int64_t ftab_cap = 0;
    int32_t *h_counters = nullptr;   // pinned, NUM_COUNTERS ints
    void *io = nullptr;              // device copies for host_io
    size_t io_bytes = 0;
    int64_t *goff = nullptr;         // device copy of the batch offsets
    size_t goff_bytes = 0;
    cudaEvent_t ev[8] = {};
    ef_stats stats = {};
    ef::Tune tune;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey;   // zero-filled in ef_ctx_create
};

namespace {

thread_local char g_err[512];

// Kernels one call launches (default wedge mode): part A 3 (+1 batched),
// f table 1, orientation (a scan of 3 + node records + 2), small wedges 4,
// class wedges 2, triangles 2 (hash tables, pair tests), finalize 1.
constexpr int64_t KERNELS_PER_CALL = 3 + 1 + 6 + 4 + 2 + 2 + 1;

void set_err(ef_ctx *c, const char *fmt, ...) {
    char *dst = c ? c->err : g_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
}

#define CU(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            set_err(ctx, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                    __LINE__);                                                              \
            return e_ == cudaErrorMemoryAllocation ? EF_ERR_OOM : EF_ERR_CUDA;              \
        }                                                                                   \
    } while (0)

#define LAUNCH(expr, what)                                       \
    do {                                                         \
        if (expr) {                                              \
            set_err(ctx, "%s launch failed: %s", what,           \
                    cudaGetErrorString(cudaGetLastError()));     \
            return EF_ERR_CUDA;                                  \
        }                                                        \
    } while (0)

inline size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

void drop_graph(ef_ctx *ctx) {
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
    memset(&ctx->gkey, 0, sizeof ctx->gkey);
}

int ensure_buffer(ef_ctx *ctx, void **buf, size_t *have, size_t need, size_t slack) {
    if (*have >= need) return EF_OK;
    if (*buf) {
        drop_graph(ctx);   // it may refer to the old buffer
        CU(cudaStreamSynchronize(ctx->stream));
        CU(cudaFree(*buf));
        *buf = nullptr;
        *have = 0;
    }
    const size_t want = need + slack;
    CU(cudaMalloc(buf, want));
    *have = want;
    return EF_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

const char *err_bits(int bits, char *buf, size_t len) {
    buf[0] = 0;
    if (bits & ef::ERRB_ROWPTR) strncat(buf, " row_ptr", len - strlen(buf) - 1);
    if (bits & ef::ERRB_RANGE) strncat(buf, " column-out-of-range", len - strlen(buf) - 1);
    if (bits & ef::ERRB_SELFLOOP) strncat(buf, " self-loop", len - strlen(buf) - 1);
    if (bits & ef::ERRB_UNSORTED) strncat(buf, " row-not-strictly-ascending", len - strlen(buf) - 1);
    if (bits & ef::ERRB_ASYM) strncat(buf, " asymmetric", len - strlen(buf) - 1);
    if (bits & ef::ERRB_CROSS) strncat(buf, " edge-between-graphs", len - strlen(buf) - 1);
    return buf;
}

int graph_error(ef_ctx *ctx, int bits) {
    char buf[192];
    set_err(ctx, "input is not a symmetric simple sorted CSR:%s", err_bits(bits, buf, sizeof buf));
    return EF_ERR_GRAPH;
}

// One graph or batch on the device (row_ptr, col_idx and outputs are device
// pointers); goff_dev / G describe a batch (nullptr / 0 for one graph).
struct Job {
    const int32_t *rp, *ci;
    int32_t n;
    int64_t m;
    const int64_t *goff_dev;
    int32_t G;
    ef_options o;
    ef_outputs out;
};

int part_a(ef_ctx *ctx, const Job &j, const ef::Scratch &s, cudaStream_t st) {
    using namespace ef;
    CU(cudaMemsetAsync(s.Tacc, 0, accumulator_bytes(s), st));
    LAUNCH(launch_prep_a(j.rp, j.ci, j.n, j.m, s, ctx->tune, st), "prep");
    if (j.goff_dev) LAUNCH(launch_batch_check(j.rp, j.ci, j.n, j.m, j.goff_dev, j.G, s, ctx->tune, st), "batch check");
    return EF_OK;
}

// Part B; with prof, events 1..7 bracket f table + orientation, small
// wedges, big wedges, hash tables, pair tests and finalize.
int part_b(ef_ctx *ctx, const Job &j, const ef::Scratch &s, int64_t fcap, bool prof, cudaStream_t st) {
    using namespace ef;
    const Tune &t = ctx->tune;
    LAUNCH(launch_ftab(s.ftab, s.tq, s.counters, fcap, st), "f table");
    LAUNCH(launch_orient(j.rp, j.ci, j.n, j.m, s, t, st), "orientation");
    if (prof) CU(cudaEventRecord(ctx->ev[2], st));
    LAUNCH(launch_wedge_small(j.rp, j.ci, s, j.o.precision, j.n, t, st), "small wedge");
    if (prof) CU(cudaEventRecord(ctx->ev[3], st));
    LAUNCH(launch_wedge_big(j.rp, j.ci, s, j.o.precision, j.o.wedge_mode, j.n, j.m, t, st), "big wedge");
    if (prof) CU(cudaEventRecord(ctx->ev[4], st));
    LAUNCH(launch_out_hash(s, j.n, j.m, t, st), "out-list hash");
    if (prof) CU(cudaEventRecord(ctx->ev[5], st));
    LAUNCH(launch_tri_pairs(s, j.n, j.m, t, st), "triangle");
    if (prof) CU(cudaEventRecord(ctx->ev[6], st));
    LAUNCH(launch_finalize(s, j.o.precision, j.n, j.out, t, st), "finalize");
    return EF_OK;
}

// Capture fn(capture stream) into the context's graph unless the cached one
// has the same key; then launch it into the context stream.
template <typename F>
int run_graph(ef_ctx *ctx, const GraphKey &key, F &&fn) {
    if (!(ctx->gexec && ctx->gkey == key)) {
        drop_graph(ctx);
        CU(cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal));
        const int rc = fn(ctx->capture);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(ctx->capture, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        CU(e);
        const cudaError_t ei = cudaGraphInstantiate(&ctx->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            ctx->gexec = nullptr;
            CU(ei);
        }
        memcpy(&ctx->gkey, &key, sizeof key);
    } else {
        ctx->stats.graph_replays += 1;
    }
    CU(cudaGraphLaunch(ctx->gexec, ctx->stream));
    return EF_OK;
}

int compute_device(ef_ctx *ctx, const Job &j) {
    using namespace ef;
    cudaStream_t st = ctx->stream;
    const ef_options &o = j.o;
    if (o.wedge_mode < 0 || o.wedge_mode > 1) {
        set_err(ctx, "wedge_mode %d is not available", o.wedge_mode);
        return EF_ERR_UNSUPPORTED;
    }
    Scratch s;
    const size_t need = carve_scratch(nullptr, j.n, j.m, s);
    int rc = ensure_buffer(ctx, &ctx->scratch, &ctx->scratch_bytes, need, need / 8);
    if (rc) return rc;
    carve_scratch((char *)ctx->scratch, j.n, j.m, s);
    const bool prof = o.profile != 0;
    const bool use_graph = o.graph != 0 && !prof;

    // f table size: from the validated max degree, else the largest possible
    int64_t fcap;
    if (o.trust_input) {
        const int64_t bound = (int64_t)j.n - 1 < j.m ? (int64_t)j.n - 1 : j.m;
        fcap = 3 * (bound > 0 ? bound : 0) + 1;
    } else {
        if (prof) CU(cudaEventRecord(ctx->ev[0], st));
        rc = part_a(ctx, j, s, st);
        if (rc) return rc;
        CU(cudaMemcpyAsync(ctx->h_counters, s.counters, NUM_COUNTERS * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        if (ctx->h_counters[CNT_ERR]) return graph_error(ctx, ctx->h_counters[CNT_ERR]);
        fcap = 3 * (int64_t)ctx->h_counters[CNT_MAXDEG] + 1;
    }
    // f table (double) followed by the fixed-point triangle corrections (int64)
    size_t have = (size_t)ctx->ftab_cap * 2 * sizeof(double);
    rc = ensure_buffer(ctx, (void **)&ctx->ftab, &have, (size_t)fcap * 2 * sizeof(double), 0);
    if (rc) return rc;
    ctx->ftab_cap = (int64_t)(have / (2 * sizeof(double)));
    s.ftab = ctx->ftab;
    s.tq = reinterpret_cast<int64_t *>(ctx->ftab + fcap);

    if (use_graph) {
        GraphKey key;
        memset(&key, 0, sizeof key);
        key.rp = j.rp;
        key.ci = j.ci;
        key.goff_dev = j.goff_dev;
        key.scratch = ctx->scratch;
        key.ftab = ctx->ftab;
        const void *outs[6] = {j.out.ef, j.out.n_clusters, j.out.s, j.out.t, j.out.triangles, j.out.flag};
        memcpy(key.outs, outs, sizeof outs);
        key.m = j.m;
        key.fcap = fcap;
        key.n = j.n;
        key.G = j.G;
        key.precision = o.precision;
        key.wedge_mode = o.wedge_mode;
        key.trust = o.trust_input;
        key.tune = ctx->tune;
        rc = run_graph(ctx, key, [&](cudaStream_t cs) {
            if (o.trust_input) {
                const int r = part_a(ctx, j, s, cs);
                if (r) return r;
            }
            return part_b(ctx, j, s, fcap, false, cs);
        });
        if (rc) return rc;
    } else {
        if (o.trust_input) {
            if (prof) CU(cudaEventRecord(ctx->ev[0], st));
            rc = part_a(ctx, j, s, st);
            if (rc) return rc;
        }
        if (prof) CU(cudaEventRecord(ctx->ev[1], st));
        rc = part_b(ctx, j, s, fcap, prof, st);
        if (rc) return rc;
        if (prof) CU(cudaEventRecord(ctx->ev[7], st));
    }
    if (!o.trust_input)
        CU(cudaMemcpyAsync(ctx->h_counters + CNT_ERR, s.counters + CNT_ERR, sizeof(int32_t), cudaMemcpyDeviceToHost,
                           st));
    return EF_OK;
}

int check_opts(ef_ctx *ctx, const ef_options &o) {
    if (o.precision != EF_PREC_FP64 && o.precision != EF_PREC_FP32C) { set_err(ctx, "bad precision %d", o.precision); return EF_ERR_ARG; }
    if (o.async && (o.host_io || !o.trust_input)) { set_err(ctx, "async needs device I/O and trust_input"); return EF_ERR_ARG; }
    return EF_OK;
}

int check_args(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m, const ef_options &o, const ef_outputs *out) {
    if (!g || !out) { set_err(ctx, "null graph or outputs"); return EF_ERR_ARG; }
    if (n < 0 || m < 0 || m >= ((int64_t)1 << 31)) { set_err(ctx, "bad sizes n=%d m=%lld", n, (long long)m); return EF_ERR_ARG; }
    if (n > 0 && (!g->row_ptr || (m > 0 && !g->col_idx))) { set_err(ctx, "null CSR array"); return EF_ERR_ARG; }
    return check_opts(ctx, o);
}

// Events: 0 start, 1 part B start (after the validation readback), 2..6
// after orientation, small wedges, big wedges, hash tables, pair tests, 7 end.
void accumulate_stats(ef_ctx *ctx, bool batched) {
    auto el = [&](int a, int b) {
        float t = 0.f;
        return cudaEventElapsedTime(&t, ctx->ev[a], ctx->ev[b]) == cudaSuccess ? (double)t : 0.0;
    };
    ef_stats &st = ctx->stats;
    st.calls += 1;
    st.prep_ms += el(0, 1);
    st.orient_ms += el(1, 2);
    st.wedge_small_ms += el(2, 3);
    st.wedge_big_ms += el(3, 4);
    st.tri_hash_ms += el(4, 5);
    st.tri_pairs_ms += el(5, 6);
    st.finalize_ms += el(6, 7);
    st.total_ms += el(0, 7);
    st.kernels += KERNELS_PER_CALL + (batched ? 1 : 0);
}

// Host I/O and synchronisation around compute_device.
int run_job(ef_ctx *ctx, Job j, const ef_outputs *host_out) {
    int rc;
    if (!j.o.host_io) {
        rc = compute_device(ctx, j);
    } else {
        // device staging: row_ptr, col_idx, then every requested output
        const size_t N = (size_t)j.n;
        size_t off = 0;
        auto place = [&](size_t bytes) { size_t o_ = off; off += al(bytes); return o_; };
        const size_t o_rp = place(4 * (N + 1)), o_ci = place(4 * (size_t)(j.m + 1));
        const size_t o_ef = place(8 * N), o_n = place(8 * N), o_s = place(8 * N), o_t = place(8 * N),
                     o_tr = place(8 * N), o_fl = place(N);
        rc = ensure_buffer(ctx, &ctx->io, &ctx->io_bytes, off, 0);
        if (rc) return rc;
        char *b = (char *)ctx->io;
        CU(cudaMemcpyAsync(b + o_rp, j.rp, 4 * (N + 1), cudaMemcpyHostToDevice, ctx->stream));
        if (j.m > 0) CU(cudaMemcpyAsync(b + o_ci, j.ci, 4 * (size_t)j.m, cudaMemcpyHostToDevice, ctx->stream));
        const ef_outputs &ho = *host_out;
        ef_outputs dout = {};
        dout.ef = ho.ef ? (double *)(b + o_ef) : nullptr;
        dout.n_clusters = ho.n_clusters ? (int64_t *)(b + o_n) : nullptr;
        dout.s = ho.s ? (int64_t *)(b + o_s) : nullptr;
        dout.t = ho.t ? (double *)(b + o_t) : nullptr;
        dout.triangles = ho.triangles ? (int64_t *)(b + o_tr) : nullptr;
        dout.flag = ho.flag ? (uint8_t *)(b + o_fl) : nullptr;
        j.rp = (const int32_t *)(b + o_rp);
        j.ci = (const int32_t *)(b + o_ci);
        j.out = dout;
        rc = compute_device(ctx, j);
        if (rc) return rc;
        if (ho.ef) CU(cudaMemcpyAsync(ho.ef, dout.ef, 8 * N, cudaMemcpyDeviceToHost, ctx->stream));
        if (ho.n_clusters) CU(cudaMemcpyAsync(ho.n_clusters, dout.n_clusters, 8 * N, cudaMemcpyDeviceToHost, ctx->stream));
        if (ho.s) CU(cudaMemcpyAsync(ho.s, dout.s, 8 * N, cudaMemcpyDeviceToHost, ctx->stream));
        if (ho.t) CU(cudaMemcpyAsync(ho.t, dout.t, 8 * N, cudaMemcpyDeviceToHost, ctx->stream));
        if (ho.triangles) CU(cudaMemcpyAsync(ho.triangles, dout.triangles, 8 * N, cudaMemcpyDeviceToHost, ctx->stream));
        if (ho.flag) CU(cudaMemcpyAsync(ho.flag, dout.flag, N, cudaMemcpyDeviceToHost, ctx->stream));
    }
    if (rc) return rc;
    if (!j.o.async) {
        CU(cudaStreamSynchronize(ctx->stream));
        if (j.o.profile) accumulate_stats(ctx, j.goff_dev != nullptr);
        if (!j.o.trust_input && ctx->h_counters[ef::CNT_ERR]) return graph_error(ctx, ctx->h_counters[ef::CNT_ERR]);
    }
    CU(cudaGetLastError());
    return EF_OK;
}

int check_tuning(ef_ctx *ctx, const ef_tuning &t) {
    if (t.row_thread_max < 1 || t.row_thread_max > ef::SMALL_MAX || t.hub_min < ef::SMALL_MAX + 1 ||
        t.hub_min > ef::MID_MAX + 1 || t.tri_variant < 0 || t.tri_variant > 1 || t.grid_per_sm < 1 ||
        t.grid_per_sm > 256) {
        set_err(ctx, "tuning out of range: row_thread_max %d (1..%d), hub_min %d (%d..%d), tri_variant %d (0..1), "
                     "grid_per_sm %d (1..256)",
                t.row_thread_max, ef::SMALL_MAX, t.hub_min, ef::SMALL_MAX + 1, ef::MID_MAX + 1, t.tri_variant,
                t.grid_per_sm);
        return EF_ERR_ARG;
    }
    return EF_OK;
}

ef_tuning to_abi(const ef::Tune &t) { return ef_tuning{t.row_thread_max, t.hub_min, t.tri_variant, t.grid_per_sm}; }

void from_abi(ef::Tune &t, const ef_tuning &a) {
    t.row_thread_max = a.row_thread_max;
    t.hub_min = a.hub_min;
    t.tri_variant = a.tri_variant;
    t.grid_per_sm = a.grid_per_sm;
}

std::mutex g_default_mu;
ef_ctx *g_default[64];

}  // namespace

namespace ef {

size_t carve_scratch(char *base, int32_t n, int64_t m, Scratch &s) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        void *p = base ? base + off : nullptr;
        off += al(bytes);
        return p;
    };
    const size_t N = (size_t)n, M = (size_t)m;
    s.D = (int32_t *)take(4 * N);
    s.sig1 = (int64_t *)take(8 * N);
    s.sig2 = (int64_t *)take(8 * N);
    s.omega = (int64_t *)take(8 * N);
    s.outdeg = (int32_t *)take(4 * N);
    s.fp_row = (uint64_t *)take(8 * N);
    s.out_ptr = (int32_t *)take(4 * (N + 1));
    s.info = (int4 *)take(16 * N);
    s.out_col = (int32_t *)take(4 * (M + 8));
    s.out_D = (int32_t *)take(4 * (M + 1));
    s.out_rng = (int2 *)take(8 * (M + 1));
    s.out_hash = (int32_t *)take(4 * (M + 8));
    s.out_src = (int32_t *)take(4 * (M + 1));
    s.Ccenter = take(8 * N);
    // accumulators that start at zero, contiguous up to the end of the counters
    // (cleared by one memset per call, see accumulator_bytes)
    s.Tacc = (double *)take(8 * N);
    s.qacc = (int64_t *)take(8 * N);
    s.tcnt = (int64_t *)take(8 * N);
    s.fp_push = (uint64_t *)take(8 * N);
    s.counters = (int32_t *)take(4 * NUM_COUNTERS);
    s.bins = (int32_t *)take(4 * N * NUM_BINS);
    s.big_chunks = (int32_t *)take(4 * (N + 1));
    s.big_partial = (double *)take(8 * (M / BIG_ROWS + N + 2));
    s.scan_tmp = (int32_t *)take(4 * (N / 4096 + 4));
    s.scan_tmp2 = (int32_t *)take(4 * (N / 4096 + 4));
    s.hub_cls = take(8 * (M + N + 2));
    s.hub_q = take(8 * (M + N + 2));
    s.hub_cidx = (int32_t *)take(4 * (M + 1));
    s.ftab = nullptr;
    return off;
}

size_t accumulator_bytes(const Scratch &s) {
    return (size_t)((const char *)(s.counters + NUM_COUNTERS) - (const char *)s.Tacc);
}

// Message for ef_last_error(NULL), for entry points that run without a context.
void set_global_error(const char *msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

}  // namespace ef

extern "C" {

int ef_ctx_create(int device, void *stream, ef_ctx **out) {
    if (!out) { set_err(nullptr, "null out pointer"); return EF_ERR_ARG; }
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        set_err(nullptr, "no CUDA device %d (count %d)", device, ndev);
        return EF_ERR_CUDA;
    }
    ef_ctx *ctx = new (std::nothrow) ef_ctx();
    if (!ctx) { set_err(nullptr, "host allocation failed"); return EF_ERR_OOM; }
    memset(&ctx->gkey, 0, sizeof ctx->gkey);
    DeviceGuard dg(device);
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    ctx->tune.num_sms = ctx->num_sms;
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_counters, ef::NUM_COUNTERS * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking);
    for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->ev[i]);
    if (e == cudaSuccess && ef::prepare_kernels()) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_err(nullptr, "context set-up failed: %s", cudaGetErrorString(e));
        ef_ctx_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? EF_ERR_OOM : EF_ERR_CUDA;
    }
    *out = ctx;
    return EF_OK;
}

int ef_ctx_destroy(ef_ctx *ctx) {
    if (!ctx) return EF_OK;
    DeviceGuard dg(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    drop_graph(ctx);
    cudaFree(ctx->scratch);
    cudaFree(ctx->ftab);
    cudaFree(ctx->io);
    cudaFree(ctx->goff);
    if (ctx->h_counters) cudaFreeHost(ctx->h_counters);
    for (int i = 0; i < 8; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    if (ctx->capture) cudaStreamDestroy(ctx->capture);
    delete ctx;
    return EF_OK;
}

const char *ef_last_error(const ef_ctx *ctx) { return ctx ? ctx->err : g_err; }

int ef_sync(ef_ctx *ctx) {
    if (!ctx) return EF_ERR_ARG;
    DeviceGuard dg(ctx->device);
    CU(cudaStreamSynchronize(ctx->stream));
    return EF_OK;
}

int ef_get_stats(ef_ctx *ctx, ef_stats *out, int reset) {
    if (!ctx || !out) return EF_ERR_ARG;
    *out = ctx->stats;
    if (reset) ctx->stats = ef_stats{};
    return EF_OK;
}

int ef_compute_ex(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m, const ef_options *opt, ef_outputs *out) {
    if (!ctx) { set_err(nullptr, "null context"); return EF_ERR_ARG; }
    ef_options o = {};
    if (opt) o = *opt;
    int rc = check_args(ctx, g, n, m, o, out);
    if (rc) return rc;
    ctx->err[0] = 0;
    if (n == 0) return EF_OK;
    DeviceGuard dg(ctx->device);
    return run_job(ctx, Job{g->row_ptr, g->col_idx, n, m, nullptr, 0, o, *out}, out);
}

int ef_compute_batched(ef_ctx *ctx, const ef_csr *g, int64_t m, const int64_t *graph_off, int32_t num_graphs,
                       const ef_options *opt, ef_outputs *out) {
    if (!ctx) { set_err(nullptr, "null context"); return EF_ERR_ARG; }
    ef_options o = {};
    if (opt) o = *opt;
    if (!graph_off || num_graphs < 1) { set_err(ctx, "null graph offsets or num_graphs < 1"); return EF_ERR_ARG; }
    if (graph_off[0] != 0) { set_err(ctx, "graph_off[0] must be 0"); return EF_ERR_ARG; }
    for (int32_t i = 0; i < num_graphs; ++i)
        if (graph_off[i + 1] < graph_off[i]) { set_err(ctx, "graph_off decreases at %d", i); return EF_ERR_ARG; }
    if (graph_off[num_graphs] >= ((int64_t)1 << 31)) { set_err(ctx, "more than 2^31-1 nodes"); return EF_ERR_ARG; }
    const int32_t n = (int32_t)graph_off[num_graphs];
    int rc = check_args(ctx, g, n, m, o, out);
    if (rc) return rc;
    ctx->err[0] = 0;
    if (n == 0) return EF_OK;
    DeviceGuard dg(ctx->device);
    const int64_t *goff_dev = nullptr;
    if (!o.trust_input) {
        // the device copy of the offsets feeds the check that no entry leaves its graph
        const size_t bytes = sizeof(int64_t) * ((size_t)num_graphs + 1);
        rc = ensure_buffer(ctx, (void **)&ctx->goff, &ctx->goff_bytes, bytes, 0);
        if (rc) return rc;
        CU(cudaMemcpyAsync(ctx->goff, graph_off, bytes, cudaMemcpyHostToDevice, ctx->stream));
        goff_dev = ctx->goff;
    }
    return run_job(ctx, Job{g->row_ptr, g->col_idx, n, m, goff_dev, num_graphs, o, *out}, out);
}

int ef_get_tuning(const ef_ctx *ctx, ef_tuning *out) {
    if (!ctx || !out) return EF_ERR_ARG;
    *out = to_abi(ctx->tune);
    return EF_OK;
}

int ef_set_tuning(ef_ctx *ctx, const ef_tuning *t) {
    if (!ctx) { set_err(nullptr, "null context"); return EF_ERR_ARG; }
    ef::Tune d;
    d.num_sms = ctx->num_sms;
    if (t) {
        const int rc = check_tuning(ctx, *t);
        if (rc) return rc;
        from_abi(d, *t);
    }
    ctx->tune = d;
    return EF_OK;
}

int ef_autotune(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m, const ef_options *opt, int32_t reps,
                ef_tuning *best) {
    if (!ctx) { set_err(nullptr, "null context"); return EF_ERR_ARG; }
    ef_options o = {};
    if (opt) o = *opt;
    if (!g || !best || reps < 1 || o.host_io) { set_err(ctx, "autotune needs a device graph, reps >= 1 and an output"); return EF_ERR_ARG; }
    ef_outputs none = {};
    int rc = check_args(ctx, g, n, m, o, &none);
    if (rc) return rc;
    if (n == 0) { *best = to_abi(ctx->tune); return EF_OK; }
    DeviceGuard dg(ctx->device);
    // the graph is validated once; the candidates then run without checks, as
    // replayed CUDA graphs, with no output but the accumulators
    o.async = 0;
    o.profile = 0;
    o.graph = 0;
    rc = run_job(ctx, Job{g->row_ptr, g->col_idx, n, m, nullptr, 0, o, none}, &none);
    if (rc) return rc;
    o.trust_input = 1;
    const ef::Tune start = ctx->tune;
    o.graph = 1;
    auto time_it = [&](double &ms) -> int {
        int r = run_job(ctx, Job{g->row_ptr, g->col_idx, n, m, nullptr, 0, o, none}, &none);   // warm-up
        if (r) return r;
        CU(cudaEventRecord(ctx->ev[0], ctx->stream));
        for (int i = 0; i < reps; ++i) {
            r = run_job(ctx, Job{g->row_ptr, g->col_idx, n, m, nullptr, 0, o, none}, &none);
            if (r) return r;
        }
        CU(cudaEventRecord(ctx->ev[7], ctx->stream));
        CU(cudaEventSynchronize(ctx->ev[7]));
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[7]));
        ms = t / reps;
        return EF_OK;
    };
    // coordinate descent, two sweeps over the knobs
    static const int rows[] = {8, 16, 32}, hubs[] = {129, 257, 513}, tris[] = {0, 1}, grids[] = {16, 32, 64, 128};
    ef::Tune cur = ctx->tune;
    double cur_ms;
    rc = time_it(cur_ms);
    if (rc) { ctx->tune = start; return rc; }
    for (int sweep = 0; sweep < 2; ++sweep) {
        for (int knob = 0; knob < 4; ++knob) {
            const int *vals = knob == 0 ? rows : knob == 1 ? hubs : knob == 2 ? tris : grids;
            const int nv = knob == 0 ? 3 : knob == 1 ? 3 : knob == 2 ? 2 : 4;
            for (int i = 0; i < nv; ++i) {
                ef::Tune cand = cur;
                int &field = knob == 0 ? cand.row_thread_max : knob == 1 ? cand.hub_min
                             : knob == 2 ? cand.tri_variant : cand.grid_per_sm;
                if (field == vals[i]) continue;
                field = vals[i];
                ctx->tune = cand;
                double ms;
                rc = time_it(ms);
                if (rc) { ctx->tune = start; return rc; }
                if (ms < cur_ms) { cur = cand; cur_ms = ms; }
            }
        }
    }
    ctx->tune = cur;
    *best = to_abi(cur);
    return EF_OK;
}

int ef_compute(const ef_csr *g, int32_t n, int64_t m, double *out_ef) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        set_err(nullptr, "no current CUDA device");
        return EF_ERR_CUDA;
    }
    ef_ctx *ctx;
    {
        std::lock_guard<std::mutex> lk(g_default_mu);
        if (!g_default[dev]) {
            int rc = ef_ctx_create(dev, nullptr, &g_default[dev]);
            if (rc) return rc;
        }
        ctx = g_default[dev];
    }
    ef_outputs out = {};
    out.ef = out_ef;
    int rc = ef_compute_ex(ctx, g, n, m, nullptr, &out);
    if (rc) snprintf(g_err, sizeof g_err, "%s", ctx->err);
    return rc;
}

}  // extern "C"
