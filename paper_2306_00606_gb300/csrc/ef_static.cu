// ef_compute_static: EF of every node without allocating any memory.
//
// Some callers cannot allocate device memory at the point where they need EF:
// code running inside a memory pool that owns the whole device, plug-ins whose
// host forbids cudaMalloc/cudaFree (which synchronise the device and can
// break its own allocator's accounting), and real-time loops that must not
// touch the allocator at all.  For them this entry point runs the same passes
// as ef_compute_ex, but on a fixed scratch area that is part of the library
// image: a file-scope __device__ array of EF_STATIC_SCRATCH_BYTES (32 MiB),
// which every GPU that loads libef holds until the process exits.
//
// Set-up: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and caches it; make that
// first call before any stream capture.  With CUDA's lazy module loading this
// lookup is also when the driver loads the module holding the array and
// reserves its 32 MiB on the device, so make the first call before a memory
// pool takes the rest of the device (a call with n = 0 does the set-up and
// nothing else).  The cached address stays valid until the device's context
// is destroyed (cudaDeviceReset); do not call this after a reset.
// Afterwards a call only launches kernels, memsets and one small
// device-to-host copy of the validation word into a stack variable.  It calls
// no cudaMalloc, cudaFree, cudaMallocHost or any other allocating routine.
//
// All calls share the one array and it keeps the previous call's contents;
// everything that must start at zero is cleared by each call.  Two calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on the array and give wrong results: serialise them.
#include "ef_internal.cuh"

#include <mutex>
#include <stdio.h>

namespace ef {
void set_global_error(const char *msg);
}

namespace {

constexpr size_t EF_STATIC_SCRATCH_BYTES = (size_t)32 << 20;

__device__ __align__(256) unsigned char g_static_scratch[EF_STATIC_SCRATCH_BYTES];

std::mutex g_static_mu;
void *g_static_addr[64];

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int fail(int code, const char *msg) {
    ef::set_global_error(msg);
    return code;
}

}  // namespace

extern "C" int ef_compute_static(const ef_csr *g, int32_t n, int64_t m, int32_t precision, double *out_ef,
                                 void *stream) {
    using namespace ef;
    if (!g || !out_ef) return fail(EF_ERR_ARG, "ef_compute_static: null graph or output");
    if (n < 0 || m < 0 || m >= ((int64_t)1 << 31)) return fail(EF_ERR_ARG, "ef_compute_static: bad sizes");
    if (precision != EF_PREC_FP64 && precision != EF_PREC_FP32C)
        return fail(EF_ERR_ARG, "ef_compute_static: bad precision");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return fail(EF_ERR_CUDA, "ef_compute_static: no current CUDA device");
    void *base;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_addr[dev]) {
            cudaError_t e = cudaGetSymbolAddress(&g_static_addr[dev], g_static_scratch);
            if (e != cudaSuccess) {
                g_static_addr[dev] = nullptr;
                cudaGetLastError();
                return fail(e == cudaErrorMemoryAllocation ? EF_ERR_OOM : EF_ERR_CUDA,
                            e == cudaErrorMemoryAllocation
                                ? "ef_compute_static: no device memory left for the fixed scratch array "
                                  "(make the first call before a memory pool takes the device)"
                                : "ef_compute_static: cudaGetSymbolAddress failed");
            }
        }
        base = g_static_addr[dev];
    }
    if (n == 0) return EF_OK;
    if (!g->row_ptr || (m > 0 && !g->col_idx)) return fail(EF_ERR_ARG, "ef_compute_static: null CSR array");

    // the f table is sized for the largest degree the graph can have
    const int64_t bound = (int64_t)n - 1 < m ? (int64_t)n - 1 : m;
    const int64_t fcap = 3 * (bound > 0 ? bound : 0) + 1;
    Scratch s;
    const size_t need = carve_scratch(nullptr, n, m, s) + al256(16 * (size_t)fcap);
    if (need > EF_STATIC_SCRATCH_BYTES) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "ef_compute_static: graph needs %zu bytes of scratch, above the fixed %zu-byte maximum "
                 "(about 172 n + 44 m + 48 min(n, m) bytes); use ef_compute_ex",
                 need, EF_STATIC_SCRATCH_BYTES);
        return fail(EF_ERR_ARG, msg);
    }

    s.ftab = (float2 *)((char *)base + carve_scratch((char *)base, n, m, s));
    s.tq = reinterpret_cast<int64_t *>(s.ftab + fcap);
    Tune t;
    if (cudaDeviceGetAttribute(&t.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        prepare_kernels())
        return fail(EF_ERR_CUDA, "ef_compute_static: device query failed");

    cudaStream_t st = (cudaStream_t)stream;
    const int32_t *rp = g->row_ptr, *ci = g->col_idx;
    if (cudaMemsetAsync(s.Tacc, 0, accumulator_bytes(s), st) != cudaSuccess)
        return fail(EF_ERR_CUDA, "ef_compute_static: memset failed");
    if (launch_prep_a(rp, ci, n, m, s, t, st))
        return fail(EF_ERR_CUDA, "ef_compute_static: prep launch failed");
    int32_t h_cnt[NUM_COUNTERS];
    if (cudaMemcpyAsync(h_cnt, s.counters, sizeof h_cnt, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(EF_ERR_CUDA, "ef_compute_static: validation readback failed");
    if (prep_error_bits(h_cnt)) return fail(EF_ERR_GRAPH, "ef_compute_static: input is not a symmetric simple sorted CSR");
    if (h_cnt[CNT_MAXDEG] > EF_MAX_DEGREE)
        return fail(EF_ERR_UNSUPPORTED, "ef_compute_static: maximum degree above EF_MAX_DEGREE (2^20)");
    const bool bins = bin_layout(t, h_cnt, n, false);
    ef_outputs out = {};
    out.ef = out_ef;
    if (launch_ftab(s.ftab, s.tq, s.counters, fcap, st) || launch_orient(rp, ci, n, m, s, t, st, nullptr, nullptr, bins) ||
        launch_wedge_small(rp, ci, s, precision, n, t, st) || launch_wedge_big(rp, ci, s, precision, 0, n, m, t, st) ||
        launch_tri_pairs(s, n, m, t, st) ||
        launch_finalize(s, precision, n, out, t, st))
        return fail(EF_ERR_CUDA, "ef_compute_static: launch failed");
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return fail(EF_ERR_CUDA, "ef_compute_static: kernel execution failed");
    return EF_OK;
}
