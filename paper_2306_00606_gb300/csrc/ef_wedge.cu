// Wedge pass of libef (Algorithm 1, Phases 1-2, open degrees).
//
// For a middle node u and an end x in N(u), the open-degree credit to x is
//     R_u(x) = sum_{j in N(u), j != x} f(D_u + D_x + D_j - 4),
// and the middle node's own credit is sum over ordered pairs = sum_x R_u(x)
// (each unordered pair (i, j) appears twice, matching the weight 2 that
// Algorithm 1 gives the middle node).  R_u(x) is written to the slot of u in
// x's row (slot rev[e] for e = (u -> x)), so every slot is written by exactly
// one thread and each node later sums its own row: no atomics.
//
// Precision modes: FP64 reads f from an FP64 table; FP32C evaluates
// d log2 d with the MUFU lg2 unit, sums in FP32 with Kahan compensation per
// thread, and converts to FP64 (times ln 2) before any cross-thread sum.
#include "ef_internal.cuh"

#include <type_traits>

namespace ef {

// ------------------------------------------------ small middle nodes (D <= 32)
// G lanes per middle node (G in {4, 8, 16, 32}); lane k owns neighbour k and
// sums f over the other neighbours of the same middle node, fetched by shuffles.
template <int G, bool F64>
__global__ void __launch_bounds__(256) k_wedge_small(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                     const int32_t *__restrict__ D, const int32_t *__restrict__ rev,
                                                     const int32_t *__restrict__ list, const int32_t *__restrict__ cnt,
                                                     int bin, const double *__restrict__ ftab, void *__restrict__ slot_,
                                                     double *__restrict__ Ccenter) {
    using Acc = typename std::conditional<F64, double, float>::type;
    Acc *slot = reinterpret_cast<Acc *>(slot_);
    constexpr int PER = 32 / G;
    const int lane = threadIdx.x & 31, grp = lane / G, k = lane % G;
    const int count = cnt[bin];
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * PER; base < count;
         base += nwarps * PER) {
        const int64_t idx = base + grp;
        const bool vc = idx < count;
        const int u = vc ? list[idx] : 0;
        const int Du = vc ? D[u] : 0;
        const int start = vc ? rp[u] : 0;
        const bool own = k < Du;
        const int e = start + k;
        const int ak = own ? D[ci[e]] : 0;
        const int b0 = Du - 4 + ak;
        Acc acc = 0;
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const int aj = __shfl_sync(FULL, ak, j, G);
            if (own && j < Du && j != k) {
                const int d = b0 + aj;  // >= 0 for D_u >= 2
                if constexpr (F64) acc += __ldg(ftab + d);
                else acc += dlog2d(fmaxf((float)d, 1.0f));
            }
        }
        double r = own ? (F64 ? (double)acc : (double)acc * LN2) : 0.0;
        if (own) slot[rev[e]] = (Acc)r;
        double c = r;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o, G);
        if (k == 0 && vc) Ccenter[u] = c;
    }
}

// ---------------------------------------------- big middle nodes, direct form
// Work item = (middle node u, chunk of BIG_ROWS neighbours).  Thread t owns
// neighbour x = chunk*BIG_ROWS + t and sums f(D_u - 4 + D_x + D_j) over all j
// in N(u), staged tile by tile in shared memory, then removes j = x.  The
// item's share of the middle-node credit goes to big_partial[item]; items are
// taken from an atomic counter (dynamic scheduling).
template <bool F64>
__global__ void __launch_bounds__(BIG_ROWS) k_wedge_big_direct(
    const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const int32_t *__restrict__ D,
    const int32_t *__restrict__ rev, const int32_t *__restrict__ list, int32_t *__restrict__ cnt,
    const int32_t *__restrict__ item_ptr, const double *__restrict__ ftab, void *__restrict__ slot_,
    double *__restrict__ partial) {
    using Acc = typename std::conditional<F64, double, float>::type;
    Acc *slot = reinterpret_cast<Acc *>(slot_);
    using Elt = typename std::conditional<F64, int, float>::type;
    __shared__ __align__(16) Elt s_a[BIG_TILE];   // FP32C: D_j as float; FP64: D_j as a table offset
    __shared__ int s_item;
    __shared__ double s_red[BIG_ROWS / 32];
    const int nb = cnt[BIN_BIG];
    const int total = item_ptr[nb];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(cnt + CNT_BIGITEM, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        int lo = 0, hi = nb - 1;   // last b with item_ptr[b] <= item
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (item_ptr[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const int u = list[lo];
        const int Du = D[u];
        const int start = rp[u];
        const int k = (item - item_ptr[lo]) * BIG_ROWS + threadIdx.x;
        const bool own = k < Du;
        const int ak = own ? D[ci[start + k]] : 0;
        const int b0 = Du - 4 + ak;
        Acc s0 = 0, s1 = 0, c0 = 0, c1 = 0;
        const Acc fb0 = (Acc)b0;
        for (int t0 = 0; t0 < Du; t0 += BIG_TILE) {
            const int tn = min(BIG_TILE, Du - t0);
            __syncthreads();
            for (int i = threadIdx.x; i < tn; i += BIG_ROWS) s_a[i] = (Elt)D[ci[start + t0 + i]];
            __syncthreads();
            if (own) {
                int i = 0;
                if constexpr (F64) {
                    for (; i + 2 <= tn; i += 2) {
                        s0 += __ldg(ftab + (b0 + s_a[i]));
                        s1 += __ldg(ftab + (b0 + s_a[i + 1]));
                    }
                    for (; i < tn; ++i) s0 += __ldg(ftab + (b0 + s_a[i]));
                } else {
                    for (; i + 4 <= tn; i += 4) {
                        const float4 q = *reinterpret_cast<const float4 *>(&s_a[i]);
                        kahan_add(s0, c0, dlog2d(fb0 + q.x));
                        kahan_add(s1, c1, dlog2d(fb0 + q.y));
                        kahan_add(s0, c0, dlog2d(fb0 + q.z));
                        kahan_add(s1, c1, dlog2d(fb0 + q.w));
                    }
                    for (; i < tn; ++i) kahan_add(s0, c0, dlog2d(fb0 + s_a[i]));
                }
            }
        }
        double r = 0.0;
        if (own) {
            if constexpr (F64) {
                r = (s0 + s1) - __ldg(ftab + (b0 + ak));
            } else {
                // d >= 31 here (D_u > 32), so no clamp is needed in d log2 d
                double sum = ((double)s0 - (double)c0) + ((double)s1 - (double)c1);
                r = (sum - (double)dlog2d(fb0 + (float)ak)) * LN2;
            }
            slot[rev[start + k]] = (Acc)r;
        }
        double t = warp_sum(r);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = t;
        __syncthreads();
        if (threadIdx.x < 32) {
            double v = threadIdx.x < BIG_ROWS / 32 ? s_red[threadIdx.x] : 0.0;
            v = warp_sum(v);
            if (threadIdx.x == 0) partial[item] = v;
        }
    }
}

// Middle-node credit of each big node: ordered sum of its items' partials.
__global__ void k_big_reduce(const int32_t *__restrict__ list, const int32_t *__restrict__ cnt,
                             const int32_t *__restrict__ item_ptr, const double *__restrict__ partial,
                             double *__restrict__ Ccenter) {
    const int nb = cnt[BIN_BIG];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        double c = 0.0;
        for (int i = item_ptr[b]; i < item_ptr[b + 1]; ++i) c += partial[i];
        Ccenter[list[b]] = c;
    }
}

template <bool F64>
static void small_all(const int32_t *rp, const int32_t *ci, const Scratch &s, int32_t n, cudaStream_t st,
                      unsigned grid) {
    const int32_t *B = s.bins;
    k_wedge_small<4, F64><<<grid, 256, 0, st>>>(rp, ci, s.D, s.rev, B + (size_t)BIN_S4 * n, s.counters, BIN_S4,
                                                s.ftab, s.slotR, s.Ccenter);
    k_wedge_small<8, F64><<<grid, 256, 0, st>>>(rp, ci, s.D, s.rev, B + (size_t)BIN_S8 * n, s.counters, BIN_S8,
                                                s.ftab, s.slotR, s.Ccenter);
    k_wedge_small<16, F64><<<grid, 256, 0, st>>>(rp, ci, s.D, s.rev, B + (size_t)BIN_S16 * n, s.counters, BIN_S16,
                                                 s.ftab, s.slotR, s.Ccenter);
    k_wedge_small<32, F64><<<grid, 256, 0, st>>>(rp, ci, s.D, s.rev, B + (size_t)BIN_S32 * n, s.counters, BIN_S32,
                                                 s.ftab, s.slotR, s.Ccenter);
}

int launch_wedge_small(const int32_t *rp, const int32_t *ci, const Scratch &s, int precision, int32_t n,
                       cudaStream_t st) {
    int64_t g = ((int64_t)n + 63) / 64;
    unsigned grid = (unsigned)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
    if (precision == EF_PREC_FP64) small_all<true>(rp, ci, s, n, st, grid);
    else small_all<false>(rp, ci, s, n, st, grid);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_wedge_big(const int32_t *rp, const int32_t *ci, const Scratch &s, int precision, int32_t n,
                     int64_t m, int num_sms, cudaStream_t st) {
    (void)m;
    const int32_t *big = s.bins + (size_t)BIN_BIG * n;
    unsigned grid = (unsigned)(num_sms * 4);
    if (precision == EF_PREC_FP64)
        k_wedge_big_direct<true><<<grid, BIG_ROWS, 0, st>>>(rp, ci, s.D, s.rev, big, s.counters, s.big_chunks, s.ftab,
                                                            s.slotR, s.big_partial);
    else
        k_wedge_big_direct<false><<<grid, BIG_ROWS, 0, st>>>(rp, ci, s.D, s.rev, big, s.counters, s.big_chunks,
                                                             s.ftab, s.slotR, s.big_partial);
    k_big_reduce<<<(unsigned)(num_sms * 2), 256, 0, st>>>(big, s.counters, s.big_chunks, s.big_partial, s.Ccenter);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
