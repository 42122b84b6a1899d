// C ABI of libef (declared in include/ef.h): contexts, scratch management,
// the orchestration of the passes, batched input, CUDA-graph replay and the
// autotuner.
//
// Pass order (one graph or one batch, all on the context stream):
//   part A   one memset of the per-node accumulators and the counters;
//            degrees + row_ptr checks + wedge bins; per-row checks,
//            sigma1/sigma2, out-degrees, the symmetry sum and (batched) the
//            check that no entry leaves its graph, in the same row pass
//   host     one small readback: validation word, symmetry sum and max
//            degree (skipped with trust_input); part B runs on valid input only
//            (device_check: no readback here; a one-thread kernel stores the
//            validation bits where every kernel of part B reads them, so part B
//            does nothing on invalid input, and the host reads the bits once
//            the call's work is done)
//   part B   f table (f(d) = d ln d and the triangle corrections, d < 3 maxdeg + 1);
//            orientation (oriented CSR + omega); wedge pass (small, then mid +
//            hub middle nodes); hash tables and pair tests; finalize (per node)
// The wedge pass and the orientation + triangle passes write disjoint
// accumulators and could run on two streams; measured on the 4M-node
// power-law graph, the concurrent form was slower (the triangle pass more
// than doubles under contention), so they run in sequence.
//
// CUDA graphs (ef_options.graph): the part that needs no host decision --
// part B, or parts A and B together under trust_input or device_check -- is
// captured once on
// a private stream and replayed into the context stream while the pointers,
// sizes, options and tuning stay the same (one cached graph per context).
#include "ef_internal.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <stdarg.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>
#include <vector>

namespace {

// What a captured graph depends on: replayed only when every byte matches
// (the layout has no padding; keys are zero-filled before use).
struct GraphKey {
    const void *rp, *ci, *goff_dev, *scratch, *ftab;
    const void *outs[6];
    int64_t m, fcap;
    int32_t n, G, precision, wedge_mode, trust, bins;
    ef::Tune tune;
    bool operator==(const GraphKey &o) const { return memcmp(this, &o, sizeof *this) == 0; }
};
static_assert(sizeof(GraphKey) == 11 * 8 + 2 * 8 + 6 * 4 + sizeof(ef::Tune), "GraphKey has padding");

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
    int32_t *h_counters = nullptr;   // pinned, NUM_COUNTERS ints, then the host copy of *d_sticky
    int32_t *d_sticky = nullptr;     // validation bits of asynchronous device-checked calls since ef_sync
    bool sticky_pending = false;     // such a call was issued since the last ef_sync
    int32_t *scratch_counters = nullptr;   // counters of the last call's scratch (device)
    void *io = nullptr;              // device copies for host_io
    size_t io_bytes = 0;
    int64_t *goff = nullptr;         // device copy of the batch offsets
    size_t goff_bytes = 0;
    cudaEvent_t ev[10] = {};   // 0-7 pass timings; 8, 9 the exact part of a ranking
    ef_stats stats = {};
    ef::Tune tune;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey;   // zero-filled in ef_ctx_create
    void *rank = nullptr;            // learned-path buffers (RankScratch)
    size_t rank_bytes = 0;
    void *acts = nullptr;            // training activations
    size_t acts_bytes = 0;
    double *dtmp = nullptr;          // small device scratch (feature sums)
    bool bins = true;                // out-lists of the current graph in degree-bin order (bin_layout)
    void *sir = nullptr;             // SIR simulation state
    size_t sir_bytes = 0;
    uint64_t mem_limit = 0;          // cap on the working buffers (0: none)
};

struct ef_model {
    int device = 0;
    ef::ModelDev *d = nullptr;
    int32_t feature_mode = 0;
    int32_t fitted = 0;
};

namespace {

thread_local char g_err[512];

// Kernels one call launches: part A 3 (the batch check runs in the row pass), f table 1, orientation
// (degree-bin layout: layout gather, a scan of 3, layout scatter; node
// layout: a scan of 3; then node records, the row kernel in two forms of
// which one returns at once, the hub rows, hash tables of the longer rows;
// the short rows' tables are filled by the row kernel itself), small wedges
// 4, big wedges (class kernels 2; direct mode: item counts, a scan of 3,
// direct kernel, reduction), pair tests 1, finalize 1; with device_check
// the validation gate 1.
int64_t kernels_per_call(bool bins, int wedge_mode, bool dev_check) {
    return 3 + 1 + (bins ? 5 : 3) + 5 + 4 + (wedge_mode == 1 ? 6 : 2) + 1 + 1 + (dev_check ? 1 : 0);
}

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

// Device bytes held in the context's working buffers.
uint64_t held_bytes(const ef_ctx *ctx) {
    return (uint64_t)ctx->scratch_bytes + (uint64_t)ctx->ftab_cap * 2 * sizeof(double) + ctx->io_bytes +
           ctx->goff_bytes + ctx->rank_bytes + ctx->acts_bytes + ctx->sir_bytes + (ctx->dtmp ? 64 * sizeof(double) : 0);
}

int ensure_buffer(ef_ctx *ctx, void **buf, size_t *have, size_t need, size_t slack) {
    if (*have >= need) return EF_OK;
    if (ctx->mem_limit) {
        // the buffer grows to need + slack, or to need alone when only that fits
        const uint64_t rest = held_bytes(ctx) - *have;
        if (rest + need > ctx->mem_limit) {
            set_err(ctx, "a buffer of %llu bytes would take the context to %llu bytes, above its memory limit "
                         "of %llu bytes", (unsigned long long)need, (unsigned long long)(rest + need),
                    (unsigned long long)ctx->mem_limit);
            return EF_ERR_OOM;
        }
        if (rest + need + slack > ctx->mem_limit) slack = 0;
    }
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

// Exact S and N need the closed forms' int64 products: every term is at most
// 6 maxdeg^3 (S_v <= N_v 3 maxdeg with N_v <= 2 maxdeg^2), below 2^63 for a
// maximum degree up to EF_MAX_DEGREE = 2^20.
int degree_limit(ef_ctx *ctx, const int32_t *h) {
    if (h[ef::CNT_MAXDEG] > EF_MAX_DEGREE) {
        set_err(ctx, "maximum degree %d is above EF_MAX_DEGREE (%d): the exact cluster-degree sums would overflow "
                     "64 bits", h[ef::CNT_MAXDEG], EF_MAX_DEGREE);
        return EF_ERR_UNSUPPORTED;
    }
    return EF_OK;
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
    LAUNCH(launch_prep_a(j.rp, j.ci, j.n, j.m, s, ctx->tune, st, j.goff_dev, j.G), "prep");
    return EF_OK;
}

// Part B; with prof, events 1..4, 6, 7 bracket f table + orientation (with
// the hash tables), small wedges, big wedges, pair tests and finalize.
int part_b(ef_ctx *ctx, const Job &j, const ef::Scratch &s, int64_t fcap, bool prof, cudaStream_t st) {
    using namespace ef;
    const Tune &t = ctx->tune;
    LAUNCH(launch_ftab(s.ftab, s.tq, s.counters, fcap, st), "f table");
    LAUNCH(launch_orient(j.rp, j.ci, j.n, j.m, s, t, st, nullptr, nullptr, ctx->bins), "orientation");
    if (prof) CU(cudaEventRecord(ctx->ev[2], st));
    LAUNCH(launch_wedge_small(j.rp, j.ci, s, j.o.precision, j.n, t, st), "small wedge");
    if (prof) CU(cudaEventRecord(ctx->ev[3], st));
    LAUNCH(launch_wedge_big(j.rp, j.ci, s, j.o.precision, j.o.wedge_mode, j.n, j.m, t, st), "big wedge");
    if (prof) CU(cudaEventRecord(ctx->ev[4], st));
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
    ctx->scratch_counters = s.counters;
    const bool prof = o.profile != 0;
    const bool use_graph = o.graph != 0 && !prof;
    const bool dev_check = o.device_check != 0 && !o.trust_input;
    // part A in the same stream as part B, with no host decision between them
    const bool a_inline = o.trust_input || dev_check;
    auto part_a_inline = [&](cudaStream_t cs) -> int {
        int r = part_a(ctx, j, s, cs);
        if (!r && dev_check) LAUNCH(launch_gate(s.counters, o.async ? ctx->d_sticky : nullptr, cs), "validation gate");
        return r;
    };

    // f table size: from the validated max degree, else the largest possible
    int64_t fcap;
    if (a_inline) {
        int64_t bound = (int64_t)j.n - 1 < j.m ? (int64_t)j.n - 1 : j.m;
        if (bound > EF_MAX_DEGREE) bound = EF_MAX_DEGREE;
        fcap = 3 * (bound > 0 ? bound : 0) + 1;
        ctx->bins = bin_layout(ctx->tune, nullptr, j.n, j.goff_dev != nullptr);
    } else {
        if (prof) CU(cudaEventRecord(ctx->ev[0], st));
        rc = part_a(ctx, j, s, st);
        if (rc) return rc;
        CU(cudaMemcpyAsync(ctx->h_counters, s.counters, NUM_COUNTERS * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        if (const int bits = prep_error_bits(ctx->h_counters)) return graph_error(ctx, bits);
        if (const int lim = degree_limit(ctx, ctx->h_counters)) return lim;
        fcap = 3 * (int64_t)ctx->h_counters[CNT_MAXDEG] + 1;
        ctx->bins = bin_layout(ctx->tune, ctx->h_counters, j.n, j.goff_dev != nullptr);
    }
    // f table (double) followed by the fixed-point triangle corrections (int64)
    size_t have = (size_t)ctx->ftab_cap * 2 * sizeof(double);
    rc = ensure_buffer(ctx, (void **)&ctx->ftab, &have, (size_t)fcap * 2 * sizeof(double), 0);
    if (rc) return rc;
    ctx->ftab_cap = (int64_t)(have / (2 * sizeof(double)));
    s.ftab = reinterpret_cast<float2 *>(ctx->ftab);
    s.tq = reinterpret_cast<int64_t *>(s.ftab + fcap);

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
        key.trust = o.trust_input | (dev_check ? 2 : 0) | (dev_check && o.async ? 4 : 0);
        key.bins = ctx->bins;
        key.tune = ctx->tune;
        rc = run_graph(ctx, key, [&](cudaStream_t cs) {
            if (a_inline) {
                const int r = part_a_inline(cs);
                if (r) return r;
            }
            return part_b(ctx, j, s, fcap, false, cs);
        });
        if (rc) return rc;
    } else {
        if (a_inline) {
            if (prof) CU(cudaEventRecord(ctx->ev[0], st));
            rc = part_a_inline(st);
            if (rc) return rc;
        }
        if (prof) CU(cudaEventRecord(ctx->ev[1], st));
        rc = part_b(ctx, j, s, fcap, prof, st);
        if (rc) return rc;
        if (prof) CU(cudaEventRecord(ctx->ev[7], st));
    }
    return EF_OK;
}

int check_opts(ef_ctx *ctx, const ef_options &o) {
    if (o.precision != EF_PREC_FP64 && o.precision != EF_PREC_FP32C) { set_err(ctx, "bad precision %d", o.precision); return EF_ERR_ARG; }
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
void accumulate_stats(ef_ctx *ctx, int wedge_mode, bool dev_check) {
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
    st.tri_pairs_ms += el(4, 6);
    st.finalize_ms += el(6, 7);
    st.total_ms += el(0, 7);
    st.kernels += kernels_per_call(ctx->bins, wedge_mode, dev_check);
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
    const bool dev_check = j.o.device_check != 0 && !j.o.trust_input;
    if (!j.o.async) {
        if (dev_check)
            CU(cudaMemcpyAsync(ctx->h_counters, ctx->scratch_counters, ef::NUM_COUNTERS * sizeof(int32_t),
                               cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        if (dev_check) {
            if (const int bits = ef::prep_error_bits(ctx->h_counters)) return graph_error(ctx, bits);
            if (const int lim = degree_limit(ctx, ctx->h_counters)) return lim;
        }
        if (j.o.profile) accumulate_stats(ctx, j.o.wedge_mode, dev_check);
    } else if (dev_check) {
        ctx->sticky_pending = true;
    }
    CU(cudaGetLastError());
    return EF_OK;
}

int check_tuning(ef_ctx *ctx, const ef_tuning &t) {
    if (t.row_thread_max < 1 || t.row_thread_max > ef::SMALL_MAX || t.hub_min < ef::SMALL_MAX + 1 ||
        t.hub_min > ef::MID_MAX + 1 || t.tri_variant < 0 || t.tri_variant > 1 || t.grid_per_sm < 1 ||
        t.grid_per_sm > 256 || t.layout < 0 || t.layout > 2) {
        set_err(ctx, "tuning out of range: row_thread_max %d (1..%d), hub_min %d (%d..%d), tri_variant %d (0..1), "
                     "grid_per_sm %d (1..256), layout %d (0..2)",
                t.row_thread_max, ef::SMALL_MAX, t.hub_min, ef::SMALL_MAX + 1, ef::MID_MAX + 1, t.tri_variant,
                t.grid_per_sm, t.layout);
        return EF_ERR_ARG;
    }
    return EF_OK;
}

ef_tuning to_abi(const ef::Tune &t) {
    return ef_tuning{t.row_thread_max, t.hub_min, t.tri_variant, t.grid_per_sm, t.layout};
}

void from_abi(ef::Tune &t, const ef_tuning &a) {
    t.row_thread_max = a.row_thread_max;
    t.hub_min = a.hub_min;
    t.tri_variant = a.tri_variant;
    t.grid_per_sm = a.grid_per_sm;
    t.layout = a.layout;
}

std::mutex g_default_mu;
ef_ctx *g_default[64];

// ----------------------------------------------------------- learned path
size_t carve_rank(char *base, int32_t n, ef::RankScratch &r) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        void *p = base ? base + off : nullptr;
        off += al(bytes);
        return p;
    };
    const size_t N = (size_t)n;
    r.x = (float *)take(4 * N * ef::MLP_F);
    r.score = (float *)take(4 * N);
    r.nbr_min = (int32_t *)take(4 * N);
    r.nbr_max = (int32_t *)take(4 * N);
    r.key = (uint64_t *)take(8 * N);
    r.flag = (int32_t *)take(4 * N);
    r.pos = (int32_t *)take(4 * (N + 1));
    r.list = (int32_t *)take(4 * N);
    r.listL = (int32_t *)take(4 * N);
    r.lista = (int32_t *)take(4 * N);
    r.role = (int32_t *)take(4 * N);
    r.hist = (int32_t *)take(4 * 65536);
    r.sel = (uint64_t *)take(8 * 4);
    r.scan_tmp = (int32_t *)take(4 * (N / 4096 + 4));
    r.exact = (double *)take(8 * N);
    r.exact_node = (double *)take(8 * N);
    r.a_score = (float *)take(4 * N);
    r.a_exact = (double *)take(8 * N);
    return off;
}

// Scratch, part A with the validation readback, and the f tables: what every
// learned-path entry needs before its own passes.
int prepare_graph(ef_ctx *ctx, const int32_t *rp, const int32_t *ci, int32_t n, int64_t m, const ef_options &o,
                  ef::Scratch &s, int64_t &fcap) {
    using namespace ef;
    const size_t need = carve_scratch(nullptr, n, m, s);
    int rc = ensure_buffer(ctx, &ctx->scratch, &ctx->scratch_bytes, need, need / 8);
    if (rc) return rc;
    carve_scratch((char *)ctx->scratch, n, m, s);
    Job j{rp, ci, n, m, nullptr, 0, o, ef_outputs{}};
    rc = part_a(ctx, j, s, ctx->stream);
    if (rc) return rc;
    if (o.trust_input) {
        const int64_t bound = (int64_t)n - 1 < m ? (int64_t)n - 1 : m;
        fcap = 3 * (bound > 0 ? bound : 0) + 1;
        ctx->bins = bin_layout(ctx->tune, nullptr, n, false);
    } else {
        CU(cudaMemcpyAsync(ctx->h_counters, s.counters, NUM_COUNTERS * sizeof(int32_t), cudaMemcpyDeviceToHost,
                           ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        if (const int bits = prep_error_bits(ctx->h_counters)) return graph_error(ctx, bits);
        if (const int lim = degree_limit(ctx, ctx->h_counters)) return lim;
        fcap = 3 * (int64_t)ctx->h_counters[CNT_MAXDEG] + 1;
        ctx->bins = bin_layout(ctx->tune, ctx->h_counters, n, false);
    }
    size_t have = (size_t)ctx->ftab_cap * 2 * sizeof(double);
    rc = ensure_buffer(ctx, (void **)&ctx->ftab, &have, (size_t)fcap * 2 * sizeof(double), 0);
    if (rc) return rc;
    ctx->ftab_cap = (int64_t)(have / (2 * sizeof(double)));
    s.ftab = reinterpret_cast<float2 *>(ctx->ftab);
    s.tq = reinterpret_cast<int64_t *>(s.ftab + fcap);
    LAUNCH(launch_ftab(s.ftab, s.tq, s.counters, fcap, ctx->stream), "f table");
    return EF_OK;
}

int rank_buffers(ef_ctx *ctx, int32_t n, ef::RankScratch &r) {
    const size_t need = carve_rank(nullptr, n, r);
    int rc = ensure_buffer(ctx, &ctx->rank, &ctx->rank_bytes, need, 0);
    if (rc) return rc;
    carve_rank((char *)ctx->rank, n, r);
    return EF_OK;
}

// Features of every node into x (after prepare_graph).  with_orient: take
// omega and the neighbour degree range from the orientation pass (which a
// ranking needs anyway for its triangles) instead of the lighter omega pass;
// the orientation always builds the hash tables, since triangles follow.
int features_device(ef_ctx *ctx, const int32_t *rp, const int32_t *ci, int32_t n, int64_t m, int mode,
                    const ef::Scratch &s, ef::RankScratch r, float *x, bool with_orient = false,
                    const ef::ModelDev *std_model = nullptr) {
    using namespace ef;
    cudaStream_t st = ctx->stream;
    if (with_orient || mode == 1)
        LAUNCH(launch_orient(rp, ci, n, m, s, ctx->tune, st, r.nbr_min, r.nbr_max, ctx->bins), "orientation");
    else
        LAUNCH(launch_omega_mm(rp, ci, n, m, s, r, ctx->tune, st), "omega");
    if (mode == 1) LAUNCH(launch_tri_pairs(s, n, m, ctx->tune, st), "triangle");
    r.x = x;
    LAUNCH(launch_features(s, r, n, mode, ctx->tune, st, std_model), "features");
    return EF_OK;
}

// Exact EF of list[0..k) (k on the device when kptr is given): the wedge
// kernels over bins of the listed nodes and their neighbours, then a CTA per
// listed node.  Triangles: per listed node (few nodes), or (global_tri) the
// full oriented triangle pass, which costs less once the list holds the
// high-EF nodes next to the hubs; orient_done / tri_done: the features
// already ran the orientation / the whole triangle pass.
int nodes_device(ef_ctx *ctx, const int32_t *rp, const int32_t *ci, int32_t n, int64_t m, const ef::Scratch &s,
                 const int32_t *list, int32_t kmax, const int32_t *kptr, int precision, bool global_tri,
                 bool orient_done, bool tri_done, const ef_outputs &out, bool timed = false) {
    using namespace ef;
    cudaStream_t st = ctx->stream;
    if (global_tri && !tri_done) {
        if (!orient_done)
            LAUNCH(launch_orient(rp, ci, n, m, s, ctx->tune, st, nullptr, nullptr, ctx->bins), "orientation");
        LAUNCH(launch_tri_pairs(s, n, m, ctx->tune, st), "triangle");
    }
    if (timed) CU(cudaEventRecord(ctx->ev[8], st));
    // the row passes' out-degrees are not needed any more: they hold the marks
    LAUNCH(launch_bin_nodes(list, kmax, kptr, rp, ci, s, s.outdeg, n, ctx->tune, st), "node bins");
    LAUNCH(launch_wedge_small(rp, ci, s, precision, n, ctx->tune, st), "small wedge");
    LAUNCH(launch_wedge_big(rp, ci, s, precision, 0, n, m, ctx->tune, st), "big wedge");
    if (timed) CU(cudaEventRecord(ctx->ev[9], st));
    LAUNCH(launch_nodes_exact(rp, ci, s, list, kmax, kptr, n, precision, global_tri, out, ctx->tune, st),
           "node exact");
    return EF_OK;
}

int final_check(ef_ctx *ctx, const ef::Scratch &s, bool validate) {
    CU(cudaMemcpyAsync(ctx->h_counters + ef::CNT_ERR, s.counters + ef::CNT_ERR, sizeof(int32_t),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    const int bits = ctx->h_counters[ef::CNT_ERR];
    if (bits & ef::ERRB_NODE) {
        set_err(ctx, "a requested node id is outside [0, n)");
        return EF_ERR_ARG;
    }
    if (validate && bits) return graph_error(ctx, bits);
    CU(cudaGetLastError());
    return EF_OK;
}

int check_learned_opts(ef_ctx *ctx, const ef_options &o) {
    int rc = check_opts(ctx, o);
    if (rc) return rc;
    if (o.host_io || o.async) { set_err(ctx, "host_io and async are not available on this entry point"); return EF_ERR_ARG; }
    return EF_OK;
}

uint64_t splitmix64(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Spearman rho with average ranks for ties (host, audit sample only).
double spearman(const std::vector<double> &a, const std::vector<double> &b) {
    const size_t n = a.size();
    if (n < 2) return 0.0;
    auto ranks = [&](const std::vector<double> &x) {
        std::vector<size_t> o(n);
        for (size_t i = 0; i < n; ++i) o[i] = i;
        std::stable_sort(o.begin(), o.end(), [&](size_t i, size_t j) { return x[i] < x[j]; });
        std::vector<double> r(n);
        for (size_t i = 0; i < n;) {
            size_t j = i;
            while (j + 1 < n && x[o[j + 1]] == x[o[i]]) ++j;
            for (size_t q = i; q <= j; ++q) r[o[q]] = (double)(i + j) / 2.0 + 1.0;
            i = j + 1;
        }
        return r;
    };
    std::vector<double> ra = ranks(a), rb = ranks(b);
    double ma = 0, mb = 0;
    for (size_t i = 0; i < n; ++i) { ma += ra[i]; mb += rb[i]; }
    ma /= n;
    mb /= n;
    double sab = 0, saa = 0, sbb = 0;
    for (size_t i = 0; i < n; ++i) {
        sab += (ra[i] - ma) * (rb[i] - mb);
        saa += (ra[i] - ma) * (ra[i] - ma);
        sbb += (rb[i] - mb) * (rb[i] - mb);
    }
    return saa > 0 && sbb > 0 ? sab / std::sqrt(saa * sbb) : 0.0;
}

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
    s.out_ptr = (int32_t *)take(4 * (N + 1));
    s.lay_node = (int32_t *)take(4 * N);
    s.lay_ptr = (int32_t *)take(4 * (N + 1));
    s.info = (int4 *)take(16 * N);
    s.out_col = (int32_t *)take(4 * (M + 8));
    s.out_D = (int32_t *)take(4 * (M + 1));
    s.out_pd = (int2 *)take(8 * (M + 1));
    s.out_hash = (int32_t *)take(4 * (M + 8));
    s.out_src = (int32_t *)take(4 * (M + 1));
    s.Ccenter = take(8 * N);
    // accumulators that start at zero, contiguous up to the end of the counters
    // (cleared by one memset per call, see accumulator_bytes)
    s.Tacc = (double *)take(8 * N);
    s.qacc = (int64_t *)take(8 * N);
    s.tcnt = (int64_t *)take(8 * N);
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
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_counters, (ef::NUM_COUNTERS + 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_sticky, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_sticky, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking);
    for (int i = 0; i < 10 && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->ev[i]);
    if (e == cudaSuccess && ef::prepare_kernels()) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_err(nullptr, "context set-up failed: %s", cudaGetErrorString(e));
        ef_ctx_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? EF_ERR_OOM : EF_ERR_CUDA;
    }
    *out = ctx;
    return EF_OK;
}

int ef_ctx_set_memory_limit(ef_ctx *ctx, uint64_t bytes) {
    if (!ctx) { set_err(nullptr, "null context"); return EF_ERR_ARG; }
    ctx->mem_limit = bytes;
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
    cudaFree(ctx->rank);
    cudaFree(ctx->acts);
    cudaFree(ctx->dtmp);
    cudaFree(ctx->sir);
    cudaFree(ctx->d_sticky);
    if (ctx->h_counters) cudaFreeHost(ctx->h_counters);
    for (int i = 0; i < 10; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    if (ctx->capture) cudaStreamDestroy(ctx->capture);
    delete ctx;
    return EF_OK;
}

const char *ef_last_error(const ef_ctx *ctx) { return ctx ? ctx->err : g_err; }

int ef_sync(ef_ctx *ctx) {
    if (!ctx) return EF_ERR_ARG;
    DeviceGuard dg(ctx->device);
    if (!ctx->sticky_pending) {
        CU(cudaStreamSynchronize(ctx->stream));
        return EF_OK;
    }
    // asynchronous device-checked calls since the last ef_sync: their
    // validation bits, OR-ed together on the device
    int32_t *h = ctx->h_counters + ef::NUM_COUNTERS;
    CU(cudaMemcpyAsync(h, ctx->d_sticky, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemsetAsync(ctx->d_sticky, 0, sizeof(int32_t), ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->sticky_pending = false;
    const int bits = *h;
    if (bits & ~ef::ERRB_DEGREE) return graph_error(ctx, bits & ~ef::ERRB_DEGREE);
    if (bits) {
        set_err(ctx, "maximum degree above EF_MAX_DEGREE (%d): the exact cluster-degree sums would overflow 64 bits",
                EF_MAX_DEGREE);
        return EF_ERR_UNSUPPORTED;
    }
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
    static const int rows[] = {8, 16, 32}, hubs[] = {129, 257, 513}, tris[] = {0, 1}, grids[] = {16, 32, 64, 128},
                     layouts[] = {1, 2};
    ef::Tune cur = ctx->tune;
    double cur_ms;
    rc = time_it(cur_ms);
    if (rc) { ctx->tune = start; return rc; }
    for (int sweep = 0; sweep < 2; ++sweep) {
        for (int knob = 0; knob < 5; ++knob) {
            const int *vals = knob == 0 ? rows : knob == 1 ? hubs : knob == 2 ? tris : knob == 3 ? grids : layouts;
            const int nv = knob == 0 ? 3 : knob == 1 ? 3 : knob == 2 ? 2 : knob == 3 ? 4 : 2;
            for (int i = 0; i < nv; ++i) {
                ef::Tune cand = cur;
                int &field = knob == 0 ? cand.row_thread_max : knob == 1 ? cand.hub_min
                             : knob == 2 ? cand.tri_variant : knob == 3 ? cand.grid_per_sm : cand.layout;
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

int ef_compute_nodes(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m, const int32_t *nodes, int32_t k,
                     const ef_options *opt, ef_outputs *out) {
    if (!ctx) { set_err(nullptr, "null context"); return EF_ERR_ARG; }
    ef_options o = {};
    if (opt) o = *opt;
    int rc = check_args(ctx, g, n, m, o, out);
    if (rc) return rc;
    rc = check_learned_opts(ctx, o);
    if (rc) return rc;
    if (k < 0 || (k > 0 && !nodes)) { set_err(ctx, "bad node list"); return EF_ERR_ARG; }
    ctx->err[0] = 0;
    if (k == 0) return EF_OK;
    if (n == 0) { set_err(ctx, "node ids given for an empty graph"); return EF_ERR_ARG; }
    DeviceGuard dg(ctx->device);
    ef::Scratch s;
    int64_t fcap;
    rc = prepare_graph(ctx, g->row_ptr, g->col_idx, n, m, o, s, fcap);
    if (rc) return rc;
    ef::RankScratch r = {};
    LAUNCH(ef::launch_omega_mm(g->row_ptr, g->col_idx, n, m, s, r, ctx->tune, ctx->stream), "omega");
    rc = nodes_device(ctx, g->row_ptr, g->col_idx, n, m, s, nodes, k, nullptr, o.precision, false, false, false,
                      *out);
    if (rc) return rc;
    return final_check(ctx, s, !o.trust_input);
}

int ef_compute_shard(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m, int32_t shard, int32_t num_shards,
                     const ef_options *opt, ef_partials *out, int32_t *frac_bits, int32_t *range) {
    using namespace ef;
    if (!ctx) { set_err(nullptr, "null context"); return EF_ERR_ARG; }
    ef_options o = {};
    if (opt) o = *opt;
    const ef_outputs none = {};
    int rc = check_args(ctx, g, n, m, o, &none);
    if (rc) return rc;
    rc = check_learned_opts(ctx, o);
    if (rc) return rc;
    if (num_shards < 1 || shard < 0 || shard >= num_shards) {
        set_err(ctx, "shard %d of %d", shard, num_shards);
        return EF_ERR_ARG;
    }
    if (!out || (n > 0 && (!out->t || !out->q || !out->triangles || !out->n_clusters || !out->s_open))) {
        set_err(ctx, "null partial array");
        return EF_ERR_ARG;
    }
    if (o.wedge_mode < 0 || o.wedge_mode > 1) {
        set_err(ctx, "wedge_mode %d is not available", o.wedge_mode);
        return EF_ERR_UNSUPPORTED;
    }
    ctx->err[0] = 0;
    if (n == 0) {
        if (frac_bits) *frac_bits = TRI_FRAC_MAX;
        if (range) memset(range, 0, 2 * sizeof(int32_t));
        return EF_OK;
    }
    DeviceGuard dg(ctx->device);
    Scratch s;
    int64_t fcap;
    rc = prepare_graph(ctx, g->row_ptr, g->col_idx, n, m, o, s, fcap);
    if (rc) return rc;
    const int32_t *rp = g->row_ptr, *ci = g->col_idx;
    const Tune &t = ctx->tune;
    cudaStream_t st = ctx->stream;
    int32_t *rng = s.counters + CNT_RANGE;
    LAUNCH(launch_shard_range(rp, n, m, shard, num_shards, rng, st), "shard range");
    LAUNCH(launch_orient(rp, ci, n, m, s, t, st, nullptr, nullptr, ctx->bins), "orientation");
    LAUNCH(launch_tri_pairs(s, n, m, t, st, rng), "triangle");
    // the out-degrees are not needed any more: they hold the marks
    LAUNCH(launch_mark_range(rng, n, s.outdeg, t, st), "shard marks");
    LAUNCH(launch_bin_marked(s.outdeg, s, n, t, st), "shard bins");
    LAUNCH(launch_wedge_small(rp, ci, s, o.precision, n, t, st), "small wedge");
    LAUNCH(launch_wedge_big(rp, ci, s, o.precision, o.wedge_mode, n, m, t, st), "big wedge");
    LAUNCH(launch_shard_out(rng, s, o.precision, n, *out, t, st), "shard partials");
    CU(cudaMemcpyAsync(ctx->h_counters + CNT_TRIFRAC, s.counters + CNT_TRIFRAC, sizeof(int32_t),
                       cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(ctx->h_counters + CNT_RANGE, rng, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    rc = final_check(ctx, s, !o.trust_input);
    if (rc) return rc;
    if (frac_bits) *frac_bits = ctx->h_counters[CNT_TRIFRAC];
    if (range) memcpy(range, ctx->h_counters + CNT_RANGE, 2 * sizeof(int32_t));
    return EF_OK;
}

int ef_finalize_partials(ef_ctx *ctx, int32_t n, const ef_partials *sum, int32_t frac_bits, const ef_options *opt,
                         ef_outputs *out) {
    using namespace ef;
    if (!ctx) { set_err(nullptr, "null context"); return EF_ERR_ARG; }
    ef_options o = {};
    if (opt) o = *opt;
    int rc = check_learned_opts(ctx, o);
    if (rc) return rc;
    if (n < 0 || !out) { set_err(ctx, "bad size n=%d or null outputs", n); return EF_ERR_ARG; }
    if (!sum || (n > 0 && (!sum->t || !sum->q || !sum->triangles || !sum->n_clusters || !sum->s_open))) {
        set_err(ctx, "null partial array");
        return EF_ERR_ARG;
    }
    if (frac_bits < 0 || frac_bits > TRI_FRAC_MAX) {
        set_err(ctx, "frac_bits %d outside 0..%d", frac_bits, TRI_FRAC_MAX);
        return EF_ERR_ARG;
    }
    ctx->err[0] = 0;
    if (n == 0) return EF_OK;
    DeviceGuard dg(ctx->device);
    LAUNCH(launch_finalize_sums(*sum, o.precision, n, frac_bits, *out, ctx->tune, ctx->stream), "finalize");
    CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaGetLastError());
    return EF_OK;
}

// Steps between two host checks of whether any simulation is still running.
constexpr int SIR_CHECK = 16;

int ef_sir_run(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m, const int32_t *index_cases, int32_t num_sims,
               const uint8_t *immune, int32_t num_immune_sets, const int32_t *immune_set,
               const ef_sir_params *params, const ef_options *opt, ef_sir_outputs *out) {
    using namespace ef;
    if (!ctx) { set_err(nullptr, "null context"); return EF_ERR_ARG; }
    ef_options o = {};
    if (opt) o = *opt;
    const ef_outputs none = {};
    int rc = check_args(ctx, g, n, m, o, &none);
    if (rc) return rc;
    rc = check_learned_opts(ctx, o);
    if (rc) return rc;
    if (!params || !out) { set_err(ctx, "null parameters or outputs"); return EF_ERR_ARG; }
    const ef_sir_params p = *params;
    if (num_sims < 0 || (num_sims > 0 && !index_cases)) { set_err(ctx, "bad simulation list"); return EF_ERR_ARG; }
    if (!(p.beta >= 0.0 && p.beta <= 1.0) || !(p.gamma >= 0.0 && p.gamma <= 1.0)) {
        set_err(ctx, "beta %g or gamma %g outside [0, 1]", p.beta, p.gamma);
        return EF_ERR_ARG;
    }
    if (p.max_steps < 1 || p.depth < 0 || p.depth > 4) {
        set_err(ctx, "max_steps %d < 1 or depth %d outside 0..4", p.max_steps, p.depth);
        return EF_ERR_ARG;
    }
    if (num_immune_sets < 0 || (num_immune_sets > 0 && !immune)) { set_err(ctx, "bad immune sets"); return EF_ERR_ARG; }
    if (out->spread && p.depth == 0) { set_err(ctx, "spread requested with depth 0"); return EF_ERR_ARG; }
    ctx->err[0] = 0;
    if (num_sims == 0) return EF_OK;
    if (n == 0) { set_err(ctx, "index cases given for an empty graph"); return EF_ERR_ARG; }
    DeviceGuard dg(ctx->device);
    Scratch s;
    int64_t fcap;
    rc = prepare_graph(ctx, g->row_ptr, g->col_idx, n, m, o, s, fcap);
    if (rc) return rc;
    cudaStream_t cs = ctx->stream;
    const Tune &t = ctx->tune;
    SirStep sp;
    sp.seed = p.seed;
    sp.beta_thr = (uint64_t)std::floor(p.beta * 4294967296.0);
    sp.gamma_thr = (uint64_t)std::floor(p.gamma * 4294967296.0);
    // state of one batch of at most SIR_BATCH simulations
    const int32_t Bmax = num_sims < SIR_BATCH ? num_sims : SIR_BATCH;
    const size_t N = (size_t)n, WBmax = ((size_t)Bmax + 31) / 32;
    size_t off = 0;
    auto place = [&](size_t bytes) { size_t o_ = off; off += al(bytes); return o_; };
    const size_t o_susc = place(4 * N * WBmax), o_inf0 = place(4 * N * WBmax), o_inf1 = place(4 * N * WBmax),
                 o_new = place(4 * N * WBmax), o_cand = place(4 * N * (size_t)Bmax),
                 o_parent = out->parent ? 0 : place(4 * N * (size_t)Bmax), o_f0 = place(4 * N), o_f1 = place(4 * N),
                 o_touch = place(4 * N), o_heavy = place(4 * N), o_fmark = place(4 * N), o_tmark = place(4 * N),
                 o_counts = place(16), o_act = place(16), o_cnt = place(4 * (size_t)Bmax),
                 o_peak = place(4 * (size_t)Bmax), o_pstep = place(4 * (size_t)Bmax), o_len = place(4 * (size_t)Bmax),
                 o_fs = place(4 * (size_t)Bmax), o_done = place((size_t)Bmax), o_err = place(4);
    rc = ensure_buffer(ctx, &ctx->sir, &ctx->sir_bytes, off, 0);
    if (rc) return rc;
    char *b = (char *)ctx->sir;
    int64_t *active = (int64_t *)(b + o_act);
    int64_t *h_active = reinterpret_cast<int64_t *>(ctx->h_counters + 48);
    if (out->spread) CU(cudaMemsetAsync(out->spread, 0, 8 * (size_t)p.depth * N, cs));
    if (out->spread_sims) CU(cudaMemsetAsync(out->spread_sims, 0, 8 * N, cs));
    for (int32_t c0 = 0; c0 < num_sims; c0 += SIR_BATCH) {
        SirState st;
        st.B = num_sims - c0 < SIR_BATCH ? num_sims - c0 : SIR_BATCH;
        st.WB = (st.B + 31) / 32;
        st.susc = (uint32_t *)(b + o_susc);
        st.inf[0] = (uint32_t *)(b + o_inf0);
        st.inf[1] = (uint32_t *)(b + o_inf1);
        st.newinf = (uint32_t *)(b + o_new);
        st.cand = (int32_t *)(b + o_cand);
        st.parent = out->parent ? out->parent + (size_t)c0 * N : (int32_t *)(b + o_parent);
        st.front[0] = (int32_t *)(b + o_f0);
        st.front[1] = (int32_t *)(b + o_f1);
        st.touched = (int32_t *)(b + o_touch);
        st.heavy = (int32_t *)(b + o_heavy);
        st.fmark = (int32_t *)(b + o_fmark);
        st.tmark = (int32_t *)(b + o_tmark);
        st.counts = (int32_t *)(b + o_counts);
        st.count = (int32_t *)(b + o_cnt);
        st.peak = (int32_t *)(b + o_peak);
        st.peak_step = (int32_t *)(b + o_pstep);
        st.length = (int32_t *)(b + o_len);
        st.fsize = (int32_t *)(b + o_fs);
        st.done = (uint8_t *)(b + o_done);
        st.err = (int32_t *)(b + o_err);
        const size_t words = 4 * N * (size_t)st.WB;
        CU(cudaMemsetAsync(st.inf[0], 0, words, cs));
        CU(cudaMemsetAsync(st.inf[1], 0, words, cs));
        CU(cudaMemsetAsync(st.newinf, 0, words, cs));
        CU(cudaMemsetAsync(st.fmark, 0, 4 * N, cs));
        CU(cudaMemsetAsync(st.tmark, 0, 4 * N, cs));
        CU(cudaMemsetAsync(st.counts, 0, 16, cs));
        CU(cudaMemsetAsync(active, 0, 16, cs));
        CU(cudaMemsetAsync(st.err, 0, sizeof(int32_t), cs));
        LAUNCH(launch_sir_init(index_cases + c0, n, immune, num_immune_sets, immune_set ? immune_set + c0 : nullptr,
                               st, t, cs),
               "SIR init");
        CU(cudaMemcpyAsync(ctx->h_counters, st.err, sizeof(int32_t), cudaMemcpyDeviceToHost, cs));
        CU(cudaStreamSynchronize(cs));
        if (ctx->h_counters[0]) {
            set_err(ctx, "an index case is outside [0, n) or immune, or an immune-set index is out of range");
            return EF_ERR_ARG;
        }
        sp.sim_base = p.sim_base + c0;
        for (int32_t step = 0; step < p.max_steps; ++step) {
            LAUNCH(launch_sir_step(g->row_ptr, g->col_idx, n, step, sp, st, active, t, cs), "SIR step");
            if ((step + 1) % SIR_CHECK == 0 && step + 1 < p.max_steps) {
                CU(cudaMemcpyAsync(h_active, active + (step & 1), sizeof(int64_t), cudaMemcpyDeviceToHost, cs));
                CU(cudaStreamSynchronize(cs));
                if (*h_active == 0) break;
            }
        }
        LAUNCH(launch_sir_close(p.max_steps, st, out->truncated ? out->truncated + c0 : nullptr, t, cs), "SIR close");
        const size_t bb = 4 * (size_t)st.B;
        if (out->final_size) CU(cudaMemcpyAsync(out->final_size + c0, st.fsize, bb, cudaMemcpyDeviceToDevice, cs));
        if (out->length) CU(cudaMemcpyAsync(out->length + c0, st.length, bb, cudaMemcpyDeviceToDevice, cs));
        if (out->peak_infected) CU(cudaMemcpyAsync(out->peak_infected + c0, st.peak, bb, cudaMemcpyDeviceToDevice, cs));
        if (out->peak_step) CU(cudaMemcpyAsync(out->peak_step + c0, st.peak_step, bb, cudaMemcpyDeviceToDevice, cs));
        if (out->spread || out->spread_sims)
            LAUNCH(launch_sir_tree(n, out->spread ? p.depth : 0, p.spread_min_size, st, out->spread, out->spread_sims,
                                   t, cs),
                   "SIR tree");
    }
    if (out->spread) LAUNCH(launch_sir_cumulate(n, p.depth, out->spread, t, cs), "SIR spread");
    CU(cudaStreamSynchronize(cs));
    CU(cudaGetLastError());
    return EF_OK;
}

int ef_features(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m, int32_t mode, const ef_options *opt, float *x) {
    if (!ctx) { set_err(nullptr, "null context"); return EF_ERR_ARG; }
    ef_options o = {};
    if (opt) o = *opt;
    ef_outputs none = {};
    int rc = check_args(ctx, g, n, m, o, &none);
    if (rc) return rc;
    rc = check_learned_opts(ctx, o);
    if (rc) return rc;
    if (mode < 0 || mode > 1 || (n > 0 && !x)) { set_err(ctx, "bad feature mode or null output"); return EF_ERR_ARG; }
    ctx->err[0] = 0;
    if (n == 0) return EF_OK;
    DeviceGuard dg(ctx->device);
    ef::Scratch s;
    int64_t fcap;
    rc = prepare_graph(ctx, g->row_ptr, g->col_idx, n, m, o, s, fcap);
    if (rc) return rc;
    ef::RankScratch r;
    rc = rank_buffers(ctx, n, r);
    if (rc) return rc;
    rc = features_device(ctx, g->row_ptr, g->col_idx, n, m, mode, s, r, x);
    if (rc) return rc;
    return final_check(ctx, s, !o.trust_input);
}

int ef_model_create(ef_ctx *ctx, uint64_t seed, int32_t feature_mode, ef_model **out) {
    if (!ctx || !out || feature_mode < 0 || feature_mode > 1) { set_err(ctx, "bad model arguments"); return EF_ERR_ARG; }
    *out = nullptr;
    DeviceGuard dg(ctx->device);
    std::vector<float> h(EF_MODEL_FLOATS, 0.f);
    uint64_t x = seed;
    auto init = [&](int off, int count, int fan_in) {
        for (int i = 0; i < count; ++i) {
            const double u = (double)(splitmix64(x) >> 11) * (1.0 / 9007199254740992.0);
            h[off + i] = (float)((2.0 * u - 1.0) / std::sqrt((double)fan_in));
        }
    };
    init(ef::P_W1, ef::MLP_F * ef::MLP_H, ef::MLP_F);
    init(ef::P_W2, ef::MLP_H * ef::MLP_H, ef::MLP_H);
    init(ef::P_W3, ef::MLP_H, ef::MLP_H);
    for (int f = 0; f < ef::MLP_F; ++f) h[ef::P_N + ef::MLP_F + f] = 1.f;   // std
    ef_model *mdl = new (std::nothrow) ef_model();
    if (!mdl) { set_err(ctx, "host allocation failed"); return EF_ERR_OOM; }
    mdl->device = ctx->device;
    mdl->feature_mode = feature_mode;
    cudaError_t e = cudaMalloc(&mdl->d, sizeof(ef::ModelDev));
    if (e == cudaSuccess) e = cudaMemset(mdl->d, 0, sizeof(ef::ModelDev));
    if (e == cudaSuccess) e = cudaMemcpy(mdl->d->p, h.data(), sizeof(float) * ef::P_N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(mdl->d->mean, h.data() + ef::P_N, sizeof(float) * 2 * ef::MLP_F, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(&mdl->d->feature_mode, &feature_mode, sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && ef::launch_model_pack(mdl->d, nullptr)) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        set_err(ctx, "model set-up failed: %s", cudaGetErrorString(e));
        cudaFree(mdl->d);
        delete mdl;
        return e == cudaErrorMemoryAllocation ? EF_ERR_OOM : EF_ERR_CUDA;
    }
    *out = mdl;
    return EF_OK;
}

int ef_model_destroy(ef_model *model) {
    if (!model) return EF_OK;
    DeviceGuard dg(model->device);
    cudaFree(model->d);
    delete model;
    return EF_OK;
}

int ef_model_feature_mode(const ef_model *model) { return model ? model->feature_mode : -1; }

int ef_model_get(const ef_model *model, float *host) {
    if (!model || !host) return EF_ERR_ARG;
    DeviceGuard dg(model->device);
    if (cudaMemcpy(host, model->d->p, sizeof(float) * ef::P_N, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(host + ef::P_N, model->d->mean, sizeof(float) * 2 * ef::MLP_F, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
        return EF_ERR_CUDA;
    return EF_OK;
}

int ef_model_set(ef_model *model, const float *host) {
    if (!model || !host) return EF_ERR_ARG;
    for (int f = 0; f < ef::MLP_F; ++f)
        if (!(host[ef::P_N + ef::MLP_F + f] > 0.f)) return EF_ERR_MODEL;   // std must be positive
    DeviceGuard dg(model->device);
    if (cudaMemcpy(model->d->p, host, sizeof(float) * ef::P_N, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(model->d->mean, host + ef::P_N, sizeof(float) * 2 * ef::MLP_F, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        ef::launch_model_pack(model->d, nullptr) || cudaDeviceSynchronize() != cudaSuccess)
        return EF_ERR_CUDA;
    model->fitted = 1;
    return EF_OK;
}

int ef_model_save(const ef_model *model, const char *path) {
    if (!model || !path) return EF_ERR_ARG;
    std::vector<float> h(EF_MODEL_FLOATS);
    int rc = ef_model_get(model, h.data());
    if (rc) return rc;
    FILE *f = fopen(path, "wb");
    if (!f) return EF_ERR_ARG;
    const char magic[8] = {'E', 'F', 'M', 'L', 'P', '0', '0', '1'};
    const int32_t hdr[2] = {model->feature_mode, model->fitted};
    const bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int32_t), 2, f) == 2 &&
                    fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
    return fclose(f) == 0 && ok ? EF_OK : EF_ERR_ARG;
}

int ef_model_load(ef_ctx *ctx, const char *path, ef_model **out) {
    if (!ctx || !path || !out) { set_err(ctx, "bad arguments"); return EF_ERR_ARG; }
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) { set_err(ctx, "cannot open %s", path); return EF_ERR_ARG; }
    char magic[8];
    int32_t hdr[2];
    std::vector<float> h(EF_MODEL_FLOATS);
    const bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "EFMLP001", 8) == 0 &&
                    fread(hdr, sizeof(int32_t), 2, f) == 2 && fread(h.data(), sizeof(float), h.size(), f) == h.size();
    fclose(f);
    if (!ok || hdr[0] < 0 || hdr[0] > 1) { set_err(ctx, "%s is not a model file", path); return EF_ERR_MODEL; }
    int rc = ef_model_create(ctx, 0, hdr[0], out);
    if (rc) return rc;
    rc = ef_model_set(*out, h.data());
    if (rc) {
        ef_model_destroy(*out);
        *out = nullptr;
        set_err(ctx, "%s holds an invalid model", path);
        return rc;
    }
    (*out)->fitted = hdr[1];
    return EF_OK;
}

int ef_mlp_forward(ef_ctx *ctx, const ef_model *model, const float *x, int32_t n, float *out) {
    if (!ctx || !model || n < 0 || (n > 0 && (!x || !out))) { set_err(ctx, "bad arguments"); return EF_ERR_ARG; }
    if (model->device != ctx->device) { set_err(ctx, "model and context on different devices"); return EF_ERR_MODEL; }
    if (n == 0) return EF_OK;
    DeviceGuard dg(ctx->device);
    LAUNCH(ef::launch_mlp_infer(model->d, x, n, out, ctx->num_sms, ctx->stream), "network");
    CU(cudaStreamSynchronize(ctx->stream));
    return EF_OK;
}

int ef_mlp_grad(ef_ctx *ctx, ef_model *model, const float *x, const float *y, int32_t n, float *loss, float *grad) {
    if (!ctx || !model || n < 1 || !x || !y || !loss || !grad) { set_err(ctx, "bad arguments"); return EF_ERR_ARG; }
    if (model->device != ctx->device) { set_err(ctx, "model and context on different devices"); return EF_ERR_MODEL; }
    DeviceGuard dg(ctx->device);
    int rc = ensure_buffer(ctx, &ctx->acts, &ctx->acts_bytes, ef::mlp_act_bytes(n), 0);
    if (rc) return rc;
    LAUNCH(ef::launch_mlp_step(model->d, x, y, n, n, 0, false, false, false, 0.f, (uint16_t *)ctx->acts,
                               ctx->num_sms, ctx->stream),
           "network gradient");
    float ls = 0.f;
    CU(cudaMemcpyAsync(grad, model->d->grad, sizeof(float) * ef::P_N, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(&ls, &model->d->loss_sum, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *loss = ls / (float)n;
    return EF_OK;
}

int ef_surrogate_train(ef_ctx *ctx, ef_model *model, const float *x, const float *y, int32_t n,
                       const ef_train_options *opt, ef_train_stats *stats) {
    if (!ctx || !model || !opt || n < 1 || !x || !y || opt->steps < 1 || opt->batch < 1 || !(opt->lr > 0.f)) {
        set_err(ctx, "bad training arguments");
        return EF_ERR_ARG;
    }
    if (model->device != ctx->device) { set_err(ctx, "model and context on different devices"); return EF_ERR_MODEL; }
    DeviceGuard dg(ctx->device);
    cudaStream_t st = ctx->stream;
    int rc = ensure_buffer(ctx, &ctx->acts, &ctx->acts_bytes, ef::mlp_act_bytes(opt->batch), 0);
    if (rc) return rc;
    if (!ctx->dtmp) CU(cudaMalloc(&ctx->dtmp, 64 * sizeof(double)));
    if (!model->fitted) {
        LAUNCH(ef::launch_feature_stats(x, n, model->d, ctx->dtmp, st), "feature statistics");
        LAUNCH(ef::launch_model_pack(model->d, st), "model pack");
        model->fitted = 1;
    }
    uint16_t *acts = (uint16_t *)ctx->acts;
    auto step = [&](cudaStream_t s) {
        return ef::launch_mlp_step(model->d, x, y, n, opt->batch, opt->seed, true, true, true, opt->lr, acts,
                                   ctx->num_sms, s);
    };
    float first = 0.f, last = 0.f;
    CU(cudaEventRecord(ctx->ev[0], st));
    LAUNCH(step(st), "training step");
    CU(cudaMemcpyAsync(&first, &model->d->loss_sum, sizeof(float), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (opt->steps > 1) {
        // the remaining steps replay one captured step (a private graph)
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        CU(cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal));
        const int lrc = step(ctx->capture);
        const cudaError_t ec = cudaStreamEndCapture(ctx->capture, &g);
        if (lrc || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            set_err(ctx, "training step capture failed");
            return EF_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        CU(ei);
        cudaError_t el = cudaSuccess;
        for (int i = 1; i < opt->steps && el == cudaSuccess; ++i) el = cudaGraphLaunch(ge, st);
        if (el == cudaSuccess) el = cudaStreamSynchronize(st);
        cudaGraphExecDestroy(ge);
        CU(el);
    }
    CU(cudaEventRecord(ctx->ev[7], st));
    CU(cudaMemcpyAsync(&last, &model->d->loss_sum, sizeof(float), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (stats) {
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[7]));
        stats->first_loss = first / (float)opt->batch;
        stats->last_loss = last / (float)opt->batch;
        stats->ms = ms;
    }
    return EF_OK;
}

int ef_surrogate_rank(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m, const ef_model *model, float top_frac,
                      float cand_frac, float audit_frac, uint64_t seed, const ef_options *opt, int32_t *out_idx,
                      double *out_ef, float *out_score, ef_rank_stats *stats) {
    using namespace ef;
    if (!ctx) { set_err(nullptr, "null context"); return EF_ERR_ARG; }
    ef_options o = {};
    if (opt) o = *opt;
    ef_outputs none = {};
    int rc = check_args(ctx, g, n, m, o, &none);
    if (rc) return rc;
    rc = check_learned_opts(ctx, o);
    if (rc) return rc;
    if (!model || !(top_frac > 0.f) || !(cand_frac >= top_frac) || cand_frac > 1.f || audit_frac < 0.f ||
        audit_frac > 1.f || n < 1) {
        set_err(ctx, "need a model, 0 < top_frac <= cand_frac <= 1, 0 <= audit_frac <= 1 and n >= 1");
        return EF_ERR_ARG;
    }
    if (model->device != ctx->device) { set_err(ctx, "model and context on different devices"); return EF_ERR_MODEL; }
    if (!model->fitted) { set_err(ctx, "the model is not trained"); return EF_ERR_MODEL; }
    ctx->err[0] = 0;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = ctx->stream;
    const int32_t kc = (int32_t)std::min<int64_t>(n, (int64_t)std::ceil((double)cand_frac * n));
    const int32_t kt = (int32_t)std::min<int64_t>(kc, (int64_t)std::ceil((double)top_frac * n));
    CU(cudaEventRecord(ctx->ev[0], st));
    Scratch s;
    int64_t fcap;
    rc = prepare_graph(ctx, g->row_ptr, g->col_idx, n, m, o, s, fcap);
    if (rc) return rc;
    RankScratch r;
    rc = rank_buffers(ctx, n, r);
    if (rc) return rc;
    // the features go out standardised and in BF16 (the network's operand),
    // half the bytes of the FP32 rows that ef_features returns
    rc = features_device(ctx, g->row_ptr, g->col_idx, n, m, model->feature_mode, s, r, r.x, true, model->d);
    if (rc) return rc;
    CU(cudaEventRecord(ctx->ev[1], st));
    LAUNCH(launch_mlp_infer_bf16(model->d, reinterpret_cast<const uint32_t *>(r.x), n, r.score, ctx->num_sms, st),
           "network");
    if (out_score) CU(cudaMemcpyAsync(out_score, r.score, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
    CU(cudaEventRecord(ctx->ev[2], st));
    // candidates, audit sample, their union
    LAUNCH(launch_keys_score(r.score, n, r.key, st), "keys");
    LAUNCH(launch_select_top(r, n, kc, 32, ctx->tune, st), "candidate selection");
    const double thr = std::ldexp((double)audit_frac, 64);
    const uint64_t threshold = audit_frac >= 1.f ? ~0ull : (uint64_t)thr;
    LAUNCH(launch_roles(r.list, kc, n, seed, threshold, r.role, st), "roles");
    LAUNCH(launch_compact_role(r.role, n, 3, r.flag, r.pos, r.scan_tmp, r.listL, st), "listing");
    const int32_t *kL = r.pos + n;   // count of listed nodes, on the device
    CU(cudaEventRecord(ctx->ev[3], st));
    ef_outputs eo = {};
    eo.ef = r.exact;
    rc = nodes_device(ctx, g->row_ptr, g->col_idx, n, m, s, r.listL, n, kL, o.precision, true, true,
                      model->feature_mode == 1, eo, stats != nullptr);
    if (rc) return rc;
    CU(cudaEventRecord(ctx->ev[4], st));
    // the reported top set: largest exact EF among the candidates
    CU(cudaMemsetAsync(r.key, 0, sizeof(uint64_t) * n, st));
    LAUNCH(launch_exact_keys(r.listL, kL, n, r.exact, r.role, r.exact_node, r.key, st), "exact keys");
    LAUNCH(launch_select_top(r, n, kt, 64, ctx->tune, st), "top selection");
    LAUNCH(launch_gather_top(r.list, kt, r.exact_node, out_idx, out_ef, st), "top set");
    // audit sample: predictions against exact EF
    LAUNCH(launch_compact_role(r.role, n, 2, r.flag, r.pos, r.scan_tmp, r.lista, st), "audit listing");
    LAUNCH(launch_gather_audit(r.lista, r.pos + n, n, r.score, r.exact_node, r.a_score, r.a_exact, st), "audit");
    CU(cudaEventRecord(ctx->ev[5], st));
    int32_t na = 0;
    CU(cudaMemcpyAsync(&na, r.pos + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    rc = final_check(ctx, s, !o.trust_input);
    if (rc) return rc;
    if (stats) {
        std::vector<float> as(na);
        std::vector<double> ae(na), ps(na);
        if (na > 0) {
            CU(cudaMemcpy(as.data(), r.a_score, sizeof(float) * na, cudaMemcpyDeviceToHost));
            CU(cudaMemcpy(ae.data(), r.a_exact, sizeof(double) * na, cudaMemcpyDeviceToHost));
        }
        double mx = 0.0;
        for (int32_t i = 0; i < na; ++i) {
            ps[i] = as[i];
            mx = std::max(mx, std::fabs(ps[i] - ae[i]));
        }
        stats->n_candidates = kc;
        stats->n_audit = na;
        stats->n_top = kt;
        stats->spearman_audit = spearman(ps, ae);
        stats->max_abs_err_audit = mx;
        float t[5];
        for (int i = 0; i < 4; ++i) CU(cudaEventElapsedTime(&t[i], ctx->ev[i], ctx->ev[i + 1]));
        CU(cudaEventElapsedTime(&t[4], ctx->ev[0], ctx->ev[5]));
        stats->features_ms = t[0];
        stats->infer_ms = t[1];
        stats->select_ms = t[2];
        stats->exact_ms = t[3];
        stats->total_ms = t[4];
        float a = 0.f, b = 0.f;
        CU(cudaEventElapsedTime(&a, ctx->ev[3], ctx->ev[8]));
        CU(cudaEventElapsedTime(&b, ctx->ev[8], ctx->ev[9]));
        stats->exact_tri_ms = a;
        stats->exact_wedge_ms = b;
    }
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
