// Finalize pass of libef (Algorithm 1, Phase 3; Eq. 1).
//
// Per node v, for every slot e of v's row (neighbour u): the slot u keeps for
// v sits at rev[e] in u's row and holds u's open-degree credit to v, the
// triangle corrections u found for v (fixed point) and their count, and
// sigma1(u).  So
//   T_v = Ccenter[v] + sum of credits + (sum of corrections + q_own[v]) 2^-F,
//   t_v = t_own[v] + sum of counts,  omega_v = sum of sigma1(u),
// and S_v and N_v are the exact integer sums of Algorithm 1's credited
// degrees and clusters, in closed form:
//   N_v = D(D-2) + sigma1,
//   S_v = D(D-1)(D-4) + 2(D-1) sigma1                      (v as middle)
//       + sigma2 - sigma1 + (D-4)(sigma1 - D) + omega - D^2 (v as an end)
//       - 8 t_v                                            (triangles)
// with D = D_v, sigma1 = sum of neighbour degrees, sigma2 = sum of their
// squares.  Then
//   EF(v) = -sum over credited clusters of (d/S) ln(d/S) = ln S - T/S,
// with EF = 0 and flag = 1 when S = 0.  A slot whose reverse was never set
// means the input was not symmetric (reported as a graph error).
//
// Precision: FP64 mode sums credits and evaluates EF in FP64.  FP32C sums
// credits in FP32 with Kahan compensation and evaluates ln S - T/S in FP32
// (absolute error a few 1e-6), except at hubs of degree > HUB_FP64_DEG where
// the final reduction and the cancellation use FP64.
//
// Rows of degree <= 32 take a thread each, 33..MID_MAX a warp, hubs a CTA.
#include "ef_internal.cuh"

namespace ef {

constexpr int HUB_FP64_DEG = 1000;

struct FinalArgs {
    const int32_t *rp, *rev;
    const int64_t *sig1, *sig2;
    const void *slots;
    const void *Ccenter;
    const int64_t *t_own, *q_own;
    int32_t *cnt;
    ef_outputs o;
};

// Per-row partial sums (credits in the accumulator precision, the rest exact).
template <bool F64>
struct Part {
    AccT<F64> ts = 0, tc = 0;   // credit sum and its Kahan compensation (FP32C)
    int64_t tt = 0, om = 0, tq = 0;
    int err = 0;
    __device__ __forceinline__ void add(const FinalArgs &f, int e) {
        const int r = f.rev[e];
        if (r < 0) {
            err |= ERRB_ASYM;
            return;
        }
        const Slot<F64> s = reinterpret_cast<const Slot<F64> *>(f.slots)[r];
        if constexpr (F64) ts += s.val;
        else kahan_add(ts, tc, s.val);
        tt += s.cnt;
        om += s.sig;
        tq += s.tri;
    }
    __device__ __forceinline__ AccT<F64> credit() const { return ts - tc; }
};

// F64: storage precision of the credits; WIDE: evaluate in FP64 (FP64 mode, or
// a hub row whose credit sum arrives already reduced in FP64).
template <bool F64, bool WIDE, typename CreditT>
__device__ __forceinline__ void finish_node(const FinalArgs &f, int v, int64_t d, CreditT credit, int64_t tt,
                                            int64_t om, int64_t tq) {
    const int64_t t = f.t_own[v] + tt;
    const int64_t qt = f.q_own[v] + tq;
    const int64_t s1 = f.sig1[v], s2 = f.sig2[v];
    const int64_t N = d * (d - 2) + s1;
    const int64_t S = d * (d - 1) * (d - 4) + 2 * (d - 1) * s1 + s2 - s1 + (d - 4) * (s1 - d) + om - d * d - 8 * t;
    const AccT<F64> cc = d >= 2 ? reinterpret_cast<const AccT<F64> *>(f.Ccenter)[v] : (AccT<F64>)0;
    double ef = 0.0, Tout;
    uint8_t fl = 1;
    if (F64 || WIDE || d > HUB_FP64_DEG) {
        const double T = (double)cc + (double)credit + ldexp((double)qt, -f.cnt[CNT_TRIFRAC]);
        Tout = T;
        if (S > 0) {
            const double Sd = (double)S;
            ef = log(Sd) - T / Sd;
            fl = 0;
        }
    } else {
        const float T = (float)cc + (float)credit + ldexpf((float)qt, -f.cnt[CNT_TRIFRAC]);
        Tout = T;
        if (S > 0) {
            // ln S = ln(m) + e ln 2 with S = m 2^e, m in [0.5, 1).  ln 2 is split
            // into 45426/2^16 (16 significant bits, so e times it is exact) plus
            // the remainder ln 2 - 45426/2^16, keeping ln S at FP32 precision.
            int e2;
            const float mant = frexpf((float)S, &e2);
            const float lnS = logf(mant) + (float)e2 * 0.693145751953125f + (float)e2 * 1.4286068203094e-06f;
            ef = (double)(lnS - __fdiv_rn(T, (float)S));
            fl = 0;
        }
    }
    const ef_outputs &o = f.o;
    if (o.ef) o.ef[v] = ef;
    if (o.n_clusters) o.n_clusters[v] = N;
    if (o.s) o.s[v] = S;
    if (o.t) o.t[v] = Tout;
    if (o.triangles) o.triangles[v] = t;
    if (o.flag) o.flag[v] = fl;
}

template <bool F64>
__global__ void __launch_bounds__(256) k_finalize(int32_t n, FinalArgs f) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    int err = 0;
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n;
         base += nwarps * 32) {
        const int v = (int)(base + lane);
        const bool in = base + lane < n;
        const int a = in ? f.rp[v] : 0, b = in ? f.rp[v + 1] : 0;
        const int Dv = b - a;
        if (in && Dv <= SMALL_MAX) {
            Part<F64> p;
#pragma unroll 4
            for (int e = a; e < b; ++e) p.add(f, e);
            err |= p.err;
            finish_node<F64, false>(f, v, Dv, p.credit(), p.tt, p.om, p.tq);
        }
        unsigned mid = __ballot_sync(FULL, in && Dv > SMALL_MAX && Dv <= MID_MAX);
        while (mid) {
            const int j = __ffs(mid) - 1;
            mid &= mid - 1;
            const int u = (int)(base + j);
            const int ua = __shfl_sync(FULL, a, j), ub = __shfl_sync(FULL, b, j);
            Part<F64> p;
            for (int e = ua + lane; e < ub; e += 32) p.add(f, e);
            err |= p.err;
            const AccT<F64> cr = warp_sum(p.credit());
            const int64_t tt = warp_sum(p.tt), om = warp_sum(p.om), tq = warp_sum(p.tq);
            if (lane == 0) finish_node<F64, false>(f, u, ub - ua, cr, tt, om, tq);
        }
    }
    err = __reduce_or_sync(FULL, err);
    if (lane == 0 && err) atomicOr(f.cnt + CNT_ERR, err);
}

// Hub rows: a CTA each; the credit sum is reduced in FP64 (FP64 work here is
// per CTA, not per slot).
template <bool F64>
__global__ void __launch_bounds__(ROW_CTA) k_finalize_hub(int32_t n, const int32_t *__restrict__ bins, FinalArgs f) {
    __shared__ double s_d[ROW_CTA / 32];
    __shared__ int64_t s_t[ROW_CTA / 32], s_o[ROW_CTA / 32], s_q[ROW_CTA / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int total = hub_total(f.cnt);
    int err = 0;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int u = hub_row(bins, n, f.cnt, it);
        const int a = f.rp[u], b = f.rp[u + 1];
        Part<F64> p;
        for (int e = a + threadIdx.x; e < b; e += ROW_CTA) p.add(f, e);
        err |= p.err;
        double cr = (double)p.credit();
        int64_t tt = p.tt, om = p.om, tq = p.tq;
        cr = warp_sum(cr);
        tt = warp_sum(tt);
        om = warp_sum(om);
        tq = warp_sum(tq);
        if (lane == 0) {
            s_d[w] = cr;
            s_t[w] = tt;
            s_o[w] = om;
            s_q[w] = tq;
        }
        __syncthreads();
        if (w == 0) {
            cr = lane < ROW_CTA / 32 ? s_d[lane] : 0.0;
            tt = lane < ROW_CTA / 32 ? s_t[lane] : 0;
            om = lane < ROW_CTA / 32 ? s_o[lane] : 0;
            tq = lane < ROW_CTA / 32 ? s_q[lane] : 0;
            cr = warp_sum(cr);
            tt = warp_sum(tt);
            om = warp_sum(om);
            tq = warp_sum(tq);
            if (lane == 0) finish_node<F64, true>(f, u, b - a, cr, tt, om, tq);
        }
        __syncthreads();
    }
    err = __reduce_or_sync(FULL, err);
    if (lane == 0 && err) atomicOr(f.cnt + CNT_ERR, err);
}

int launch_finalize(const int32_t *rp, const int32_t *ci, const Scratch &s, int precision, int32_t n,
                    const ef_outputs &out, int num_sms, cudaStream_t st) {
    (void)ci;
    FinalArgs f{rp, s.rev, s.sig1, s.sig2, s.slot, s.Ccenter, s.t_own, s.q_own, s.counters, out};
    int64_t g = ((int64_t)n + 255) / 256;
    unsigned grid = (unsigned)(g < 1 ? 1 : (g > num_sms * 64 ? num_sms * 64 : g));
    if (precision == EF_PREC_FP64) {
        k_finalize<true><<<grid, 256, 0, st>>>(n, f);
        k_finalize_hub<true><<<num_sms * 4, ROW_CTA, 0, st>>>(n, s.bins, f);
    } else {
        k_finalize<false><<<grid, 256, 0, st>>>(n, f);
        k_finalize_hub<false><<<num_sms * 4, ROW_CTA, 0, st>>>(n, s.bins, f);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
