// Wedge pass of libef (Algorithm 1, Phases 1-2, open degrees).
//
// For a middle node u and an end x in N(u), the open-degree credit to x is
//     R_u(x) = sum_{j in N(u), j != x} f(D_u + D_x + D_j - 4),
// and the middle node's own credit is sum over ordered pairs = sum_x R_u(x)
// (each unordered pair (i, j) appears twice, matching the weight 2 that
// Algorithm 1 gives the middle node).  The middle node's credit is reduced
// in registers and stored once (Ccenter[u]); R_u(x) is added to x's
// accumulator Tacc[x] by an FP64 reduction in L2 (RED, no return value).
//
// Precision modes: FP64 reads f from a table computed in FP64 and held as
// FP32 pairs, and sums rows in FP32-pair chunks (F2Sum, below 2^-38 relative
// error per chunk) added up in FP64; FP32C evaluates d log2 d with the MUFU
// lg2 unit and sums in FP32 with Kahan compensation per thread (times ln 2
// at the end); the end credits travel as FP64 in both.
#include "ef_internal.cuh"

#include <type_traits>

namespace ef {

// ------------------------------------------------ small middle nodes (D <= 32)
// G lanes per middle node (G in {4, 8, 16, 32}); lane k owns neighbour k and
// sums f over the other neighbours of the same middle node, fetched by
// shuffles.  Measured and left out: summing over the node's degree classes
// (lanes of equal D_x found with one 64-bit match, class leaders' degrees
// and counts shuffled in), although the 4096-graph WS batch has 6x fewer
// distinct (degree, degree) pairs than ordered neighbour pairs: small wedges
// 3.50 -> 4.44 ms there, 0.30 -> 0.51 ms on the power-law graph (the match
// and two indexed shuffles per class cost more than the pairs they save).
//
// A warp step takes SMALL_ILP sets of 32 / G rows and issues their chains of
// dependent loads (work list -> degree and row start -> neighbour -> its
// degree) together.  FP32C, small wedges (ms) with 1 / 2 / 3 sets: WS batch
// 3.25 / 2.93 / 2.92, BA 16M 2.83 / 2.82 / 2.73, power-law 4M 0.283 / 0.286 /
// 0.288; three sets take 37-40 registers instead of 32.
constexpr int SMALL_ILP = 2;

template <int G, bool F64>
__global__ void __launch_bounds__(256) k_wedge_small(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                     const int32_t *__restrict__ D, const int32_t *__restrict__ list,
                                                     const int32_t *__restrict__ cnt, int bin,
                                                     const float2 *__restrict__ ftab, double *__restrict__ Tacc,
                                                     void *__restrict__ Ccenter) {
    if (gate_closed(cnt)) return;
    using Acc = typename std::conditional<F64, double, float>::type;
    constexpr int PER = 32 / G, ILP = SMALL_ILP;
    const int lane = threadIdx.x & 31, grp = lane / G, k = lane % G;
    const int count = cnt[bin];
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * PER * ILP; base0 < count;
         base0 += nwarps * PER * ILP) {
        int us[ILP], Dus[ILP], xs[ILP], aks[ILP];
#pragma unroll
        for (int r = 0; r < ILP; ++r) {
            const int64_t idx = base0 + r * PER + grp;
            us[r] = idx < count ? list[idx] : -1;
        }
        int sts[ILP];
#pragma unroll
        for (int r = 0; r < ILP; ++r) {
            Dus[r] = us[r] >= 0 ? D[us[r]] : 0;
            sts[r] = us[r] >= 0 ? rp[us[r]] : 0;
        }
#pragma unroll
        for (int r = 0; r < ILP; ++r) xs[r] = k < Dus[r] ? ci[sts[r] + k] : 0;
#pragma unroll
        for (int r = 0; r < ILP; ++r) aks[r] = k < Dus[r] ? D[xs[r]] : 0;
#pragma unroll
        for (int r = 0; r < ILP; ++r) {
            const bool vc = us[r] >= 0;
            const int u = vc ? us[r] : 0;
            const int Du = Dus[r];
            const bool own = k < Du;
            const int x = xs[r];
            const int ak = aks[r];
            const int b0 = Du - 4 + ak;
            Acc acc = 0;
            // the warp's largest row bounds the loop (rows of a bin are often
            // much shorter than G); degrees travel as floats (exact below 2^24),
            // so no conversion sits in the loop
            const int jmax = __reduce_max_sync(FULL, Du);
            if constexpr (F64) {
                // at most 31 terms: one FP32-pair chunk (F2Sum)
                F2Sum a2;
#pragma unroll 4
                for (int j = 0; j < jmax; ++j) {
                    const int aj = __shfl_sync(FULL, ak, j, G);
                    if (own && j < Du && j != k) a2.add(__ldg(ftab + (b0 + aj)));   // b0 + aj >= 0 for D_u >= 2
                }
                acc = a2.value();
            } else {
                // One FMA per term.  Up to the warp's shortest row every lane's
                // terms are real, so that loop adds without a test; the rest of
                // the rows (jmin..jmax) add under j < D_u.  Both include the
                // lane's own term j = k once, removed at the end (one of D_u
                // positive terms).  d = D_u - 4 + D_x + D_j >= 3 once D_u > 4
                // (G >= 8): only the smallest bin needs the guard that keeps d = 0
                // from 0 * log2(0)
                const float akf = (float)ak, b0f = (float)b0;
                const int jmin = __reduce_min_sync(FULL, vc ? Du : G);
                const int lim = own ? Du : 0;
                float sum = 0.0f;
#pragma unroll 4
                for (int j = 0; j < jmin; ++j) {
                    float d = b0f + __shfl_sync(FULL, akf, j, G);
                    if (G == 4) d = fmaxf(d, 1.0f);
                    sum = fmaf(d, __log2f(d), sum);
                }
                for (int j = jmin; j < jmax; ++j) {
                    float d = b0f + __shfl_sync(FULL, akf, j, G);
                    if (G == 4) d = fmaxf(d, 1.0f);
                    const float t = __log2f(d);
                    if (j < lim) sum = fmaf(d, t, sum);
                }
                acc = sum - dlog2d(G == 4 ? fmaxf(b0f + akf, 1.0f) : b0f + akf);
            }
            const Acc rs = own ? (F64 ? acc : acc * (Acc)LN2) : (Acc)0;
            if (own) credit_end(Tacc, x, (double)rs);
            const Acc c = group_sum<G>(rs);
            if (k == 0 && vc) reinterpret_cast<Acc *>(Ccenter)[u] = c;
        }
    }
}

// ---------------------------------------------- big middle nodes, direct form
// Work item = (middle node u, chunk of BIG_ROWS neighbours).  Thread t owns
// neighbour x = chunk*BIG_ROWS + t and sums f(D_u - 4 + D_x + D_j) over all j
// in N(u), staged tile by tile in shared memory, then removes j = x.  The
// item's share of the middle-node credit goes to big_partial[item]; items are
// taken from an atomic counter (dynamic scheduling).  This is the plain
// pairwise form, kept as the reference kernel (wedge_mode 1).
template <bool F64>
__global__ void __launch_bounds__(BIG_ROWS) k_wedge_big_direct(
    const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const int32_t *__restrict__ D,
    const int32_t *__restrict__ list, int32_t *__restrict__ cnt, const int32_t *__restrict__ item_ptr,
    const float2 *__restrict__ ftab, double *__restrict__ Tacc, double *__restrict__ partial) {
    if (gate_closed(cnt)) return;
    using Acc = typename std::conditional<F64, double, float>::type;
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
        const int x = own ? ci[start + k] : 0;
        const int ak = own ? D[x] : 0;
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
                        s0 += f2_value(__ldg(ftab + (b0 + s_a[i])));
                        s1 += f2_value(__ldg(ftab + (b0 + s_a[i + 1])));
                    }
                    for (; i < tn; ++i) s0 += f2_value(__ldg(ftab + (b0 + s_a[i])));
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
                r = (s0 + s1) - f2_value(__ldg(ftab + (b0 + ak)));
            } else {
                // d >= 31 here (D_u > 32), so no clamp is needed in d log2 d
                double sum = ((double)s0 - (double)c0) + ((double)s1 - (double)c1);
                r = (sum - (double)dlog2d(fb0 + (float)ak)) * LN2;
            }
            credit_end(Tacc, x, r);
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
template <bool F64>
__global__ void k_big_reduce(const int32_t *__restrict__ list, const int32_t *__restrict__ cnt,
                             const int32_t *__restrict__ item_ptr, const double *__restrict__ partial,
                             void *__restrict__ Ccenter_) {
    if (gate_closed(cnt)) return;
    AccT<F64> *Ccenter = reinterpret_cast<AccT<F64> *>(Ccenter_);
    const int nb = cnt[BIN_BIG];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        double c = 0.0;
        for (int i = item_ptr[b]; i < item_ptr[b + 1]; ++i) c += partial[i];
        Ccenter[list[b]] = (AccT<F64>)c;
    }
}

// ------------------------------------------------- degree-class wedge kernels
// For a middle node u, R_u(x) depends on its end x only through D_x:
//     R_u(x) = Q_u(D_x) - f(D_u - 4 + 2 D_x),
//     Q_u(a) = sum_b c_u(b) f(D_u - 4 + a + b),
// where c_u(b) is the number of neighbours of u of degree b, and the middle
// node's credit is sum_a c_u(a) R_u(a).  So u costs K_u^2 evaluations of f
// (K_u = distinct neighbour degrees) instead of D_u^2.  The classes are
// found with a dense histogram over small degrees plus one class per
// neighbour of large degree (duplicates among those stay separate classes:
// still exact, only a little redundant work).

// Per-class arithmetic: FP32C keeps (degree, count) as floats and sums
// count * d log2 d with Kahan compensation; FP64 keeps them as ints and sums
// count * f(d) from the FP64 table.
template <bool F64>
struct ClassEval;

template <>
struct ClassEval<false> {
    using Cls = float2;
    using R = float;
    static __device__ __forceinline__ Cls make(int b, int c, bool = true) { return make_float2((float)b, (float)c); }
    static __device__ __forceinline__ float bval(Cls x) { return x.x; }
    static __device__ __forceinline__ float cval(Cls x, bool = true) { return x.y; }
    // returns R = (sum_j c_j f(base + b_i + b_j) - f(base + 2 b_i)) in natural-log units.
    // Chunks of CHUNK classes are summed in plain FP32 (every term is >= 0,
    // so a chunk's rounding error is below CHUNK ulps of its sum) and the
    // chunk sums with Kahan compensation: one FMA per class pair instead of
    // a multiply and a four-operation compensated add.
    static constexpr int CHUNK = 8;
    static __device__ __forceinline__ float row(const Cls *cls, int K, int base, Cls ci, const float2 *,
                                                bool = true) {
        const float fb = (float)base + ci.x;
        float s = 0.f, c = 0.f;
        int j = 0;
        for (; j + CHUNK <= K; j += CHUNK) {
            float t0 = 0.f, t1 = 0.f;
#pragma unroll
            for (int q = 0; q < CHUNK; q += 2) {
                const float4 v = *reinterpret_cast<const float4 *>(cls + j + q);
                t0 = fmaf(v.y, dlog2d(fb + v.x), t0);
                t1 = fmaf(v.w, dlog2d(fb + v.z), t1);
            }
            kahan_add(s, c, t0 + t1);
        }
        float t = 0.f;
        for (; j < K; ++j) t = fmaf(cls[j].y, dlog2d(fb + cls[j].x), t);
        kahan_add(s, c, t);
        return ((s - c) - dlog2d(fb + ci.x)) * (float)LN2;
    }
};

template <>
struct ClassEval<true> {
    // (degree, count): the count as FP32 bits when it is exact in FP32
    // (pair_ok: the middle node's degree is below 2^24), else as an int
    using Cls = int2;
    using R = double;
    static __device__ __forceinline__ Cls make(int b, int c, bool pair_ok = true) {
        return make_int2(b, pair_ok ? __float_as_int((float)c) : c);
    }
    static __device__ __forceinline__ int bval(Cls x) { return x.x; }
    static __device__ __forceinline__ double cval(Cls x, bool pair_ok = true) {
        return pair_ok ? (double)__int_as_float(x.y) : (double)x.y;
    }
    // The row in FP32-pair chunks of F2_CHUNK classes (F2Sum), the chunk sums
    // in FP64 (pair_ok), else every term an FP64 FMA.
    static __device__ __forceinline__ double row(const Cls *cls, int K, int base, Cls ci, const float2 *ftab,
                                                 bool pair_ok = true) {
        const int fb = base + ci.x;
        double s = 0.0;
        if (pair_ok) {
            int j = 0;
            while (j < K) {
                const int je = min(K, j + F2_CHUNK);
                F2Sum a, b;
                for (; j + 2 <= je; j += 2) {
                    const int4 q = *reinterpret_cast<const int4 *>(cls + j);
                    a.add(__ldg(ftab + (fb + q.x)), __int_as_float(q.y));
                    b.add(__ldg(ftab + (fb + q.z)), __int_as_float(q.w));
                }
                if (j < je) {
                    a.add(__ldg(ftab + (fb + cls[j].x)), __int_as_float(cls[j].y));
                    ++j;
                }
                s += a.value() + b.value();
            }
        } else {
            for (int j = 0; j < K; ++j) s = fma((double)cls[j].y, f2_value(__ldg(ftab + (fb + cls[j].x))), s);
        }
        return s - f2_value(__ldg(ftab + (fb + ci.x)));
    }
};

constexpr int MID_WARPS = 4;

// One warp per middle node of degree 33..MID_MAX.  Warps take their nodes
// one at a time from an atomic counter (the work of a node grows with the
// square of its class count, which varies a hundredfold within the bin); the
// next node's index, id and row range are loaded while the current node is
// processed, so only the neighbour gathers wait at the start of a node.
template <bool F64>
__global__ void __launch_bounds__(MID_WARPS * 32) k_wedge_mid(
    const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const int32_t *__restrict__ D,
    const int32_t *__restrict__ list, int32_t *__restrict__ cnt, const float2 *__restrict__ ftab,
    double *__restrict__ Tacc, void *__restrict__ Ccenter) {
    if (gate_closed(cnt)) return;
    using E = ClassEval<F64>;
    using Cls = typename E::Cls;
    using R = typename E::R;
    __shared__ int32_t s_hist[MID_WARPS][MID_HIST];
    __shared__ int32_t s_cidx[MID_WARPS][MID_MAX];
    __shared__ __align__(16) Cls s_cls[MID_WARPS][MID_MAX];
    __shared__ R s_q[MID_WARPS][MID_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t *hist = s_hist[w], *cidx = s_cidx[w];
    Cls *cls = s_cls[w];
    R *cq = s_q[w];
    const unsigned lt = (1u << lane) - 1u;
    const int count = cnt[BIN_MID];
    int it = 0;
    if (lane == 0) it = atomicAdd(cnt + CNT_MIDITEM, 1);
    it = __shfl_sync(FULL, it, 0);
    int u = 0, start = 0, Du = 0;
    if (it < count) {
        u = list[it];
        start = rp[u];
        Du = rp[u + 1] - start;
    }
    while (it < count) {
        int next = 0;
        if (lane == 0) next = atomicAdd(cnt + CNT_MIDITEM, 1);
        const int base = Du - 4;
        for (int i = lane; i < MID_HIST; i += 32) hist[i] = 0;
        __syncwarp();
        for (int k = lane; k < Du; k += 32) {
            const int a = D[ci[start + k]];
            cidx[k] = a;
            if (a < MID_HIST) atomicAdd(hist + a, 1);
        }
        __syncwarp();
        next = __shfl_sync(FULL, next, 0);
        const int u_next = next < count ? list[next] : 0;
        int K = 0;
        for (int i0 = 0; i0 < MID_HIST; i0 += 32) {
            const int i = i0 + lane;
            const int c = hist[i];
            const unsigned bal = __ballot_sync(FULL, c > 0);
            if (c > 0) {
                const int idx = K + __popc(bal & lt);
                cls[idx] = E::make(i, c);
                hist[i] = idx;
            }
            K += __popc(bal);
        }
        __syncwarp();
        for (int k0 = 0; k0 < Du; k0 += 32) {
            const int k = k0 + lane;
            const bool act = k < Du;
            const int a = act ? cidx[k] : 0;
            const bool sp = act && a >= MID_HIST;
            const unsigned bal = __ballot_sync(FULL, sp);
            if (sp) {
                const int idx = K + __popc(bal & lt);
                cls[idx] = E::make(a, 1);
                cidx[k] = idx;
            } else if (act) {
                cidx[k] = hist[a];
            }
            K += __popc(bal);
        }
        __syncwarp();
        const int start_next = next < count ? rp[u_next] : 0;
        const int end_next = next < count ? rp[u_next + 1] : 0;
        SumAcc<R> center;
        for (int i = lane; i < K; i += 32) {
            const Cls c_i = cls[i];
            const R r = E::row(cls, K, base, c_i, ftab);
            cq[i] = r;
            center.add((R)E::cval(c_i) * r);
        }
        __syncwarp();
        for (int k = lane; k < Du; k += 32) credit_end(Tacc, ci[start + k], (double)cq[cidx[k]]);
        const R ctot = warp_sum(center.get());
        if (lane == 0) reinterpret_cast<R *>(Ccenter)[u] = ctot;
        __syncwarp();
        it = next;
        u = u_next;
        start = start_next;
        Du = end_next - start_next;
    }
}

// Block-wide exclusive scan of one int per thread (HUB_THREADS threads).
__device__ __forceinline__ int hub_scan(int x, int *s_w, int &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int t = lane < HUB_THREADS / 32 ? s_w[lane] : 0;
        int ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, ti, o);
            if (lane >= o) ti += y;
        }
        s_w[lane] = ti - t;
        if (lane == 31) s_w[32] = ti;
    }
    __syncthreads();
    const int r = s_w[w] + inc - x;
    total = s_w[32];
    __syncthreads();
    return r;
}

// One CTA per hub (degree > MID_MAX), hubs taken largest degree bucket first
// from an atomic counter.  Global arrays hold the class index of every
// neighbour (cidx_g, at the hub's own row positions) and, for hubs with more
// than HUB_SMEM_K classes, the classes themselves (cls_g, q_g).
template <bool F64>
__global__ void __launch_bounds__(HUB_THREADS) k_wedge_hub(
    const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const int32_t *__restrict__ D,
    const int32_t *__restrict__ bins, int32_t n, int32_t *__restrict__ cnt, const float2 *__restrict__ ftab,
    double *__restrict__ Tacc, void *__restrict__ Ccenter, int32_t *__restrict__ cidx_g, void *__restrict__ cls_g_,
    void *__restrict__ q_g_) {
    if (gate_closed(cnt)) return;
    using E = ClassEval<F64>;
    using Cls = typename E::Cls;
    using R = typename E::R;
    Cls *cls_g = reinterpret_cast<Cls *>(cls_g_);
    R *q_g = reinterpret_cast<R *>(q_g_);
    extern __shared__ __align__(16) unsigned char hub_smem[];
    int32_t *hist = reinterpret_cast<int32_t *>(hub_smem);
    Cls *cls_s = reinterpret_cast<Cls *>(hub_smem + HUB_HIST * sizeof(int32_t));
    R *q_s = reinterpret_cast<R *>(hub_smem + HUB_HIST * sizeof(int32_t) + HUB_SMEM_K * sizeof(Cls));
    __shared__ int s_w[33];
    __shared__ int s_item, s_nsp, s_kb;
    __shared__ double s_red[HUB_THREADS / 32];
    const int tid = threadIdx.x;
    int total = 0;
    for (int b = NUM_HUB_BUCKETS - 1; b >= 0; --b) total += cnt[BIN_HUB0 + b];
    for (;;) {
        if (tid == 0) s_item = atomicAdd(cnt + CNT_HUB, 1);
        __syncthreads();
        int item = s_item;
        if (item >= total) break;
        int b = NUM_HUB_BUCKETS - 1;
        while (item >= cnt[BIN_HUB0 + b]) item -= cnt[BIN_HUB0 + b--];
        const int u = bins[(size_t)(BIN_HUB0 + b) * n + item];
        const int start = rp[u];
        const int Du = rp[u + 1] - start;
        const int base = Du - 4;
        const bool pair_ok = Du < (1 << 24);   // class counts exact in FP32 (FP64 mode)
        int32_t *cidx = cidx_g + start;
        for (int i = tid; i < HUB_HIST; i += HUB_THREADS) hist[i] = 0;
        if (tid == 0) s_nsp = 0;
        __syncthreads();
        int nsp = 0;
        for (int k = tid; k < Du; k += HUB_THREADS) {
            const int a = D[ci[start + k]];
            cidx[k] = a;
            if (a < HUB_HIST) atomicAdd(hist + a, 1);
            else ++nsp;
        }
        nsp = __reduce_add_sync(FULL, nsp);
        if ((tid & 31) == 0 && nsp) atomicAdd(&s_nsp, nsp);
        __syncthreads();
        // dense classes: thread t owns bins [4t, 4t+4)
        int hc[HUB_HIST / HUB_THREADS];
        int mine = 0;
#pragma unroll
        for (int j = 0; j < HUB_HIST / HUB_THREADS; ++j) {
            hc[j] = hist[tid * (HUB_HIST / HUB_THREADS) + j];
            mine += hc[j] > 0;
        }
        int Kd;
        int off = hub_scan(mine, s_w, Kd);
        const int K = Kd + s_nsp;
        // global fallback: rows own disjoint ranges [start + u, start + u + Du], and an
        // even first index keeps the pairwise 16-byte class loads aligned
        const int64_t gpos = ((int64_t)start + u + 1) & ~(int64_t)1;
        Cls *cls = K <= HUB_SMEM_K ? cls_s : cls_g + gpos;
        R *cq = K <= HUB_SMEM_K ? q_s : q_g + gpos;
#pragma unroll
        for (int j = 0; j < HUB_HIST / HUB_THREADS; ++j) {
            const int bin = tid * (HUB_HIST / HUB_THREADS) + j;
            if (hc[j] > 0) {
                cls[off] = E::make(bin, hc[j], pair_ok);
                hist[bin] = off++;
            }
        }
        if (tid == 0) s_kb = Kd;
        __syncthreads();
        // sparse classes: positions from a shared counter, one atomic per warp
        // and pass (no block barrier inside the loop; their order varies)
        const unsigned lt = (1u << (tid & 31)) - 1u;
        for (int k0 = 0; k0 < Du; k0 += HUB_THREADS) {
            const int k = k0 + tid;
            const bool act = k < Du;
            const int a = act ? cidx[k] : 0;
            const bool sp = act && a >= HUB_HIST;
            const unsigned bal = __ballot_sync(FULL, sp);
            int wbase = 0;
            if ((tid & 31) == 0 && bal) wbase = atomicAdd(&s_kb, __popc(bal));
            wbase = __shfl_sync(FULL, wbase, 0);
            if (sp) {
                const int pos = wbase + __popc(bal & lt);
                cls[pos] = E::make(a, 1, pair_ok);
                cidx[k] = pos;
            } else if (act) {
                cidx[k] = hist[a];
            }
        }
        __syncthreads();
        double center = 0.0;
        for (int i = tid; i < K; i += HUB_THREADS) {
            const Cls c_i = cls[i];
            const R r = E::row(cls, K, base, c_i, ftab, pair_ok);
            cq[i] = r;
            center += (double)E::cval(c_i, pair_ok) * (double)r;
        }
        __syncthreads();
        for (int k = tid; k < Du; k += HUB_THREADS) credit_end(Tacc, ci[start + k], (double)cq[cidx[k]]);
        center = warp_sum(center);
        if ((tid & 31) == 0) s_red[tid >> 5] = center;
        __syncthreads();
        if (tid < 32) {
            double v = tid < HUB_THREADS / 32 ? s_red[tid] : 0.0;
            v = warp_sum(v);
            if (tid == 0) reinterpret_cast<R *>(Ccenter)[u] = (R)v;
        }
    }
}


template <bool F64>
static void small_all(const int32_t *rp, const int32_t *ci, const Scratch &s, int32_t n, cudaStream_t st,
                      unsigned grid) {
    const int32_t *B = s.bins;
    k_wedge_small<4, F64><<<grid, 256, 0, st>>>(rp, ci, s.D, B + (size_t)BIN_S4 * n, s.counters, BIN_S4, s.ftab,
                                                s.Tacc, s.Ccenter);
    k_wedge_small<8, F64><<<grid, 256, 0, st>>>(rp, ci, s.D, B + (size_t)BIN_S8 * n, s.counters, BIN_S8, s.ftab,
                                                s.Tacc, s.Ccenter);
    k_wedge_small<16, F64><<<grid, 256, 0, st>>>(rp, ci, s.D, B + (size_t)BIN_S16 * n, s.counters, BIN_S16, s.ftab,
                                                 s.Tacc, s.Ccenter);
    k_wedge_small<32, F64><<<grid, 256, 0, st>>>(rp, ci, s.D, B + (size_t)BIN_S32 * n, s.counters, BIN_S32, s.ftab,
                                                 s.Tacc, s.Ccenter);
}

int launch_wedge_small(const int32_t *rp, const int32_t *ci, const Scratch &s, int precision, int32_t n,
                       const Tune &t, cudaStream_t st) {
    int64_t g = ((int64_t)n + 63) / 64;
    const int64_t cap = (int64_t)t.num_sms * 16;
    unsigned grid = (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
    if (precision == EF_PREC_FP64) small_all<true>(rp, ci, s, n, st, grid);
    else small_all<false>(rp, ci, s, n, st, grid);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <bool F64>
static size_t hub_smem_bytes() {
    using E = ClassEval<F64>;
    return HUB_HIST * sizeof(int32_t) + HUB_SMEM_K * (sizeof(typename E::Cls) + sizeof(typename E::R));
}

// Per device (kept per device id, so that a process using several devices
// of different kinds sizes each one's grids from its own properties):
// resident blocks per SM of the class kernels ([F64][mid, hub]), whose grids
// hold exactly one wave while their warps take work from atomic counters,
// and the L2 size.
constexpr int MAX_DEVICES = 64;
struct DeviceProps {
    int class_blocks[2][2] = {{1, 1}, {1, 1}};
    int64_t l2_bytes = 0;
};
static DeviceProps g_dev_props[MAX_DEVICES];

static DeviceProps &dev_props() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) dev = 0;
    return g_dev_props[dev];
}

template <bool F64>
static int class_occupancy(DeviceProps &p) {
    int mid = 0, hub = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&mid, k_wedge_mid<F64>, MID_WARPS * 32, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&hub, k_wedge_hub<F64>, HUB_THREADS, hub_smem_bytes<F64>()) !=
            cudaSuccess)
        return -1;
    p.class_blocks[F64][0] = mid > 0 ? mid : 1;
    p.class_blocks[F64][1] = hub > 0 ? hub : 1;
    return 0;
}

// L2 size of the current device (read by prepare_kernels).
int64_t device_l2_bytes() { return dev_props().l2_bytes; }

// Opt the hub kernels in to their dynamic shared memory on the current device,
// size the class kernels' grids and read the L2 size (once per context,
// before any launch or stream capture).
int prepare_kernels() {
    if (cudaFuncSetAttribute(k_wedge_hub<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)hub_smem_bytes<true>()) != cudaSuccess ||
        cudaFuncSetAttribute(k_wedge_hub<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)hub_smem_bytes<false>()) != cudaSuccess)
        return -1;
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
        return -1;
    DeviceProps &p = g_dev_props[dev];
    if (class_occupancy<true>(p) || class_occupancy<false>(p) || prepare_final_tables()) return -1;
    p.l2_bytes = l2;
    return 0;
}

template <bool F64>
static int big_classes(const int32_t *rp, const int32_t *ci, const Scratch &s, int32_t n, int num_sms,
                       cudaStream_t st) {
    const int32_t *mid = s.bins + (size_t)BIN_MID * n;
    const DeviceProps &p = dev_props();
    k_wedge_mid<F64><<<(unsigned)(num_sms * p.class_blocks[F64][0]), MID_WARPS * 32, 0, st>>>(
        rp, ci, s.D, mid, s.counters, s.ftab, s.Tacc, s.Ccenter);
    const size_t smem = hub_smem_bytes<F64>();
    k_wedge_hub<F64><<<(unsigned)(num_sms * p.class_blocks[F64][1]), HUB_THREADS, smem, st>>>(
        rp, ci, s.D, s.bins, n, s.counters, s.ftab, s.Tacc, s.Ccenter, s.hub_cidx, s.hub_cls, s.hub_q);
    return 0;
}

int launch_wedge_big(const int32_t *rp, const int32_t *ci, const Scratch &s, int precision, int wedge_mode,
                     int32_t n, int64_t m, const Tune &t, cudaStream_t st) {
    (void)m;
    const int num_sms = t.num_sms;
    const int32_t *big = s.bins + (size_t)BIN_BIG * n;
    if (wedge_mode == 1) {
        if (launch_big_items(s, n, st)) return -1;
        unsigned grid = (unsigned)(num_sms * 4);
        if (precision == EF_PREC_FP64) {
            k_wedge_big_direct<true><<<grid, BIG_ROWS, 0, st>>>(rp, ci, s.D, big, s.counters, s.big_chunks, s.ftab,
                                                                s.Tacc, s.big_partial);
            k_big_reduce<true><<<(unsigned)(num_sms * 2), 256, 0, st>>>(big, s.counters, s.big_chunks,
                                                                        s.big_partial, s.Ccenter);
        } else {
            k_wedge_big_direct<false><<<grid, BIG_ROWS, 0, st>>>(rp, ci, s.D, big, s.counters, s.big_chunks, s.ftab,
                                                                 s.Tacc, s.big_partial);
            k_big_reduce<false><<<(unsigned)(num_sms * 2), 256, 0, st>>>(big, s.counters, s.big_chunks,
                                                                         s.big_partial, s.Ccenter);
        }
    } else {
        int rc = precision == EF_PREC_FP64 ? big_classes<true>(rp, ci, s, n, num_sms, st)
                                           : big_classes<false>(rp, ci, s, n, num_sms, st);
        if (rc) return rc;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
