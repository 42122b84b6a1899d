// C ABI of libef (declared in include/ef.h): contexts, scratch management and
// the orchestration of the passes for one graph.
//
// Pass order (one graph, all on the context stream):
//   one memset of the per-node accumulators and the counters
//   prep A       degrees + row_ptr checks + wedge bins; per-row checks,
//                sigma1/sigma2, out-degrees, symmetry fingerprints
//   host         one small readback: validation word and max degree
//                (skipped with trust_input)
//   f table      f(d) = d ln d and the triangle corrections, d < 3 maxdeg + 1
//   orientation  oriented CSR + omega
//   wedge pass   small, then mid + hub middle nodes
//   triangles    pair tests and corrections
//   finalize     per node
//   host         final readback of the validation word (asymmetric input is
//                only detected by the finalize pass)
// The wedge pass and the orientation + triangle passes write disjoint
// accumulators and could run on two streams; measured on the 4M-node
// power-law graph, the concurrent form was slower (the triangle pass more
// than doubles under contention), so they run in sequence.
#include "ef_internal.cuh"

#include <mutex>
#include <new>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

struct ef_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    char err[512] = {0};
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    double *ftab = nullptr;
    int64_t ftab_cap = 0;
    int32_t *h_counters = nullptr;   // pinned, NUM_COUNTERS ints
    void *io = nullptr;              // device copies for host_io
    size_t io_bytes = 0;
    cudaEvent_t ev[8] = {};
    ef_stats stats = {};
};

namespace {

thread_local char g_err[512];

// Kernels one ef_compute_ex call launches (default wedge mode): prep A 3,
// f table 1, orientation (a scan of 3 + 2), small wedges 4, class wedges 2,
// triangles 2 (hash tables, pair tests), finalize 1.
constexpr int64_t KERNELS_PER_CALL = 3 + 1 + 5 + 4 + 2 + 2 + 1;

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

int ensure_buffer(ef_ctx *ctx, void **buf, size_t *have, size_t need, size_t slack) {
    if (*have >= need) return EF_OK;
    if (*buf) {
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
    return buf;
}

int graph_error(ef_ctx *ctx, int bits) {
    char buf[160];
    set_err(ctx, "input is not a symmetric simple sorted CSR:%s", err_bits(bits, buf, sizeof buf));
    return EF_ERR_GRAPH;
}

int compute_device(ef_ctx *ctx, const int32_t *rp, const int32_t *ci, int32_t n, int64_t m, const ef_options &o,
                   const ef_outputs &out) {
    using namespace ef;
    cudaStream_t st = ctx->stream;
    if (o.wedge_mode < 0 || o.wedge_mode > 1) {
        set_err(ctx, "wedge_mode %d is not available", o.wedge_mode);
        return EF_ERR_UNSUPPORTED;
    }
    Scratch s;
    const size_t need = carve_scratch(nullptr, n, m, s);
    int rc = ensure_buffer(ctx, &ctx->scratch, &ctx->scratch_bytes, need, need / 8);
    if (rc) return rc;
    carve_scratch((char *)ctx->scratch, n, m, s);
    const bool prof = o.profile != 0;
    if (prof) CU(cudaEventRecord(ctx->ev[0], st));

    CU(cudaMemsetAsync(s.Tacc, 0, accumulator_bytes(s), st));
    LAUNCH(launch_prep_a(rp, ci, n, m, s, st), "prep");

    int64_t fcap;
    if (!o.trust_input) {
        CU(cudaMemcpyAsync(ctx->h_counters, s.counters, NUM_COUNTERS * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        if (ctx->h_counters[CNT_ERR]) return graph_error(ctx, ctx->h_counters[CNT_ERR]);
        fcap = 3 * (int64_t)ctx->h_counters[CNT_MAXDEG] + 1;
    } else {
        const int64_t bound = (int64_t)n - 1 < m ? (int64_t)n - 1 : m;
        fcap = 3 * (bound > 0 ? bound : 0) + 1;
    }
    // f table (double) followed by the fixed-point triangle corrections (int64)
    size_t have = (size_t)ctx->ftab_cap * 2 * sizeof(double);
    rc = ensure_buffer(ctx, (void **)&ctx->ftab, &have, (size_t)fcap * 2 * sizeof(double), 0);
    if (rc) return rc;
    ctx->ftab_cap = (int64_t)(have / (2 * sizeof(double)));
    s.ftab = ctx->ftab;
    s.tq = reinterpret_cast<int64_t *>(ctx->ftab + fcap);
    LAUNCH(launch_ftab(s.ftab, s.tq, s.counters, fcap, st), "f table");
    if (prof) CU(cudaEventRecord(ctx->ev[1], st));
    LAUNCH(launch_orient(rp, ci, n, m, s, st), "orientation");
    if (prof) CU(cudaEventRecord(ctx->ev[2], st));
    LAUNCH(launch_wedge_small(rp, ci, s, o.precision, n, st), "small wedge");
    if (prof) CU(cudaEventRecord(ctx->ev[3], st));
    LAUNCH(launch_wedge_big(rp, ci, s, o.precision, o.wedge_mode, n, m, ctx->num_sms, st), "big wedge");
    if (prof) CU(cudaEventRecord(ctx->ev[4], st));
    LAUNCH(launch_out_hash(s, n, m, ctx->num_sms, st), "out-list hash");
    if (prof) CU(cudaEventRecord(ctx->ev[5], st));
    LAUNCH(launch_tri_pairs(s, n, m, ctx->num_sms, st), "triangle");
    if (prof) CU(cudaEventRecord(ctx->ev[6], st));
    LAUNCH(launch_finalize(s, o.precision, n, out, ctx->num_sms, st), "finalize");
    if (prof) CU(cudaEventRecord(ctx->ev[7], st));
    if (!o.trust_input)
        CU(cudaMemcpyAsync(ctx->h_counters + CNT_ERR, s.counters + CNT_ERR, sizeof(int32_t), cudaMemcpyDeviceToHost,
                           st));
    return EF_OK;
}

int check_args(ef_ctx *ctx, const ef_csr *g, int32_t n, int64_t m, const ef_options &o, const ef_outputs *out) {
    if (!g || !out) { set_err(ctx, "null graph or outputs"); return EF_ERR_ARG; }
    if (n < 0 || m < 0 || m >= ((int64_t)1 << 31)) { set_err(ctx, "bad sizes n=%d m=%lld", n, (long long)m); return EF_ERR_ARG; }
    if (n > 0 && (!g->row_ptr || (m > 0 && !g->col_idx))) { set_err(ctx, "null CSR array"); return EF_ERR_ARG; }
    if (o.precision != EF_PREC_FP64 && o.precision != EF_PREC_FP32C) { set_err(ctx, "bad precision %d", o.precision); return EF_ERR_ARG; }
    if (o.async && (o.host_io || !o.trust_input)) { set_err(ctx, "async needs device I/O and trust_input"); return EF_ERR_ARG; }
    return EF_OK;
}

// Events 0..7 bracket, in order: prep + f table, orientation, small wedges,
// big wedges, hash tables, pair tests, finalize.
void accumulate_stats(ef_ctx *ctx) {
    float t[7], tot;
    for (int i = 0; i < 7; ++i)
        if (cudaEventElapsedTime(&t[i], ctx->ev[i], ctx->ev[i + 1]) != cudaSuccess) t[i] = 0.f;
    if (cudaEventElapsedTime(&tot, ctx->ev[0], ctx->ev[7]) != cudaSuccess) tot = 0.f;
    ef_stats &st = ctx->stats;
    st.calls += 1;
    st.prep_ms += t[0];
    st.orient_ms += t[1];
    st.wedge_small_ms += t[2];
    st.wedge_big_ms += t[3];
    st.tri_hash_ms += t[4];
    st.tri_pairs_ms += t[5];
    st.finalize_ms += t[6];
    st.total_ms += tot;
    st.kernels += KERNELS_PER_CALL;
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
    DeviceGuard dg(device);
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_counters, ef::NUM_COUNTERS * sizeof(int32_t));
    for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->ev[i]);
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
    cudaFree(ctx->scratch);
    cudaFree(ctx->ftab);
    cudaFree(ctx->io);
    if (ctx->h_counters) cudaFreeHost(ctx->h_counters);
    for (int i = 0; i < 8; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
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
    if (!o.host_io) {
        rc = compute_device(ctx, g->row_ptr, g->col_idx, n, m, o, *out);
    } else {
        // device staging: row_ptr, col_idx, then every requested output
        const size_t N = (size_t)n;
        size_t off = 0;
        auto place = [&](size_t bytes) { size_t o_ = off; off += al(bytes); return o_; };
        const size_t o_rp = place(4 * (N + 1)), o_ci = place(4 * (size_t)(m + 1));
        const size_t o_ef = place(8 * N), o_n = place(8 * N), o_s = place(8 * N), o_t = place(8 * N),
                     o_tr = place(8 * N), o_fl = place(N);
        rc = ensure_buffer(ctx, &ctx->io, &ctx->io_bytes, off, 0);
        if (rc) return rc;
        char *b = (char *)ctx->io;
        CU(cudaMemcpyAsync(b + o_rp, g->row_ptr, 4 * (N + 1), cudaMemcpyHostToDevice, ctx->stream));
        if (m > 0) CU(cudaMemcpyAsync(b + o_ci, g->col_idx, 4 * (size_t)m, cudaMemcpyHostToDevice, ctx->stream));
        ef_outputs dout = {};
        dout.ef = out->ef ? (double *)(b + o_ef) : nullptr;
        dout.n_clusters = out->n_clusters ? (int64_t *)(b + o_n) : nullptr;
        dout.s = out->s ? (int64_t *)(b + o_s) : nullptr;
        dout.t = out->t ? (double *)(b + o_t) : nullptr;
        dout.triangles = out->triangles ? (int64_t *)(b + o_tr) : nullptr;
        dout.flag = out->flag ? (uint8_t *)(b + o_fl) : nullptr;
        rc = compute_device(ctx, (const int32_t *)(b + o_rp), (const int32_t *)(b + o_ci), n, m, o, dout);
        if (rc) return rc;
        if (out->ef) CU(cudaMemcpyAsync(out->ef, dout.ef, 8 * N, cudaMemcpyDeviceToHost, ctx->stream));
        if (out->n_clusters) CU(cudaMemcpyAsync(out->n_clusters, dout.n_clusters, 8 * N, cudaMemcpyDeviceToHost, ctx->stream));
        if (out->s) CU(cudaMemcpyAsync(out->s, dout.s, 8 * N, cudaMemcpyDeviceToHost, ctx->stream));
        if (out->t) CU(cudaMemcpyAsync(out->t, dout.t, 8 * N, cudaMemcpyDeviceToHost, ctx->stream));
        if (out->triangles) CU(cudaMemcpyAsync(out->triangles, dout.triangles, 8 * N, cudaMemcpyDeviceToHost, ctx->stream));
        if (out->flag) CU(cudaMemcpyAsync(out->flag, dout.flag, N, cudaMemcpyDeviceToHost, ctx->stream));
    }
    if (rc) return rc;
    if (!o.async) {
        CU(cudaStreamSynchronize(ctx->stream));
        if (o.profile) accumulate_stats(ctx);
        if (!o.trust_input && ctx->h_counters[ef::CNT_ERR]) return graph_error(ctx, ctx->h_counters[ef::CNT_ERR]);
    }
    CU(cudaGetLastError());
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
