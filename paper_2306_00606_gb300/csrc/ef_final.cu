// Finalize pass of libef (Algorithm 1, Phase 3; Eq. 1).
//
// Per node v: T_v = Ccenter[v] (its middle-node credit and the triangle
// corrections it found as owner) + the sum of the slots of v's row (open-
// degree credits and triangle corrections from every neighbour); t_v the
// same way from the count slots.  S_v and N_v are the exact integer sums of
// Algorithm 1's credited degrees and clusters, in closed form:
//   N_v = D(D-2) + sigma1,
//   S_v = D(D-1)(D-4) + 2(D-1) sigma1                      (v as middle)
//       + sigma2 - sigma1 + (D-4)(sigma1 - D) + omega - D^2 (v as an end)
//       - 8 t_v                                            (triangles)
// with D = D_v, sigma1 = sum of neighbour degrees, sigma2 = sum of their
// squares and omega = sum of the neighbours' sigma1.  Then
//   EF(v) = -sum over credited clusters of (d/S) ln(d/S) = ln S - T/S,
// with EF = 0 and flag = 1 when S = 0.
//
// Rows of degree <= 32 take a thread each, 33..MID_MAX a warp, hubs a CTA.
#include "ef_internal.cuh"

#include <type_traits>

namespace ef {

__device__ __forceinline__ void finish_node(int v, int64_t d, double tsum, int64_t tt, int64_t om,
                                            const int64_t *__restrict__ sig1, const int64_t *__restrict__ sig2,
                                            const double *__restrict__ Ccenter, const int64_t *__restrict__ t_own,
                                            const ef_outputs &o) {
    const int64_t t = t_own[v] + tt;
    const double T = (d >= 2 ? Ccenter[v] : 0.0) + tsum;
    const int64_t s1 = sig1[v], s2 = sig2[v];
    const int64_t N = d * (d - 2) + s1;
    const int64_t S = d * (d - 1) * (d - 4) + 2 * (d - 1) * s1 + s2 - s1 + (d - 4) * (s1 - d) + om - d * d - 8 * t;
    double ef = 0.0;
    uint8_t fl = 1;
    if (S > 0) {
        const double Sd = (double)S;
        ef = log(Sd) - T / Sd;
        fl = 0;
    }
    if (o.ef) o.ef[v] = ef;
    if (o.n_clusters) o.n_clusters[v] = N;
    if (o.s) o.s[v] = S;
    if (o.t) o.t[v] = T;
    if (o.triangles) o.triangles[v] = t;
    if (o.flag) o.flag[v] = fl;
}

struct FinalArgs {
    const int32_t *rp, *ci;
    const int64_t *sig1, *sig2;
    const void *slot;
    const int32_t *slotT;
    const double *Ccenter;
    const int64_t *t_own;
    ef_outputs o;
};

template <bool F64>
__device__ __forceinline__ void row_part(const FinalArgs &f, int e, double &ts, int64_t &tt, int64_t &om) {
    using Acc = typename std::conditional<F64, double, float>::type;
    ts += (double)reinterpret_cast<const Acc *>(f.slot)[e];
    tt += f.slotT[e];
    om += f.sig1[f.ci[e]];
}

template <bool F64>
__global__ void __launch_bounds__(256) k_finalize(int32_t n, FinalArgs f) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n;
         base += nwarps * 32) {
        const int v = (int)(base + lane);
        const bool in = base + lane < n;
        const int a = in ? f.rp[v] : 0, b = in ? f.rp[v + 1] : 0;
        const int Dv = b - a;
        if (in && Dv <= SMALL_MAX) {
            double ts = 0.0;
            int64_t tt = 0, om = 0;
            for (int e = a; e < b; ++e) row_part<F64>(f, e, ts, tt, om);
            finish_node(v, Dv, ts, tt, om, f.sig1, f.sig2, f.Ccenter, f.t_own, f.o);
        }
        unsigned mid = __ballot_sync(FULL, in && Dv > SMALL_MAX && Dv <= MID_MAX);
        while (mid) {
            const int j = __ffs(mid) - 1;
            mid &= mid - 1;
            const int u = (int)(base + j);
            const int ua = __shfl_sync(FULL, a, j), ub = __shfl_sync(FULL, b, j);
            double ts = 0.0;
            int64_t tt = 0, om = 0;
            for (int e = ua + lane; e < ub; e += 32) row_part<F64>(f, e, ts, tt, om);
            ts = warp_sum(ts);
            tt = warp_sum(tt);
            om = warp_sum(om);
            if (lane == 0) finish_node(u, ub - ua, ts, tt, om, f.sig1, f.sig2, f.Ccenter, f.t_own, f.o);
        }
    }
}

template <bool F64>
__global__ void __launch_bounds__(ROW_CTA) k_finalize_hub(int32_t n, const int32_t *__restrict__ bins,
                                                          const int32_t *__restrict__ cnt, FinalArgs f) {
    __shared__ double s_d[ROW_CTA / 32];
    __shared__ int64_t s_t[ROW_CTA / 32], s_o[ROW_CTA / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int total = hub_total(cnt);
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int u = hub_row(bins, n, cnt, it);
        const int a = f.rp[u], b = f.rp[u + 1];
        double ts = 0.0;
        int64_t tt = 0, om = 0;
        for (int e = a + threadIdx.x; e < b; e += ROW_CTA) row_part<F64>(f, e, ts, tt, om);
        ts = warp_sum(ts);
        tt = warp_sum(tt);
        om = warp_sum(om);
        if (lane == 0) {
            s_d[w] = ts;
            s_t[w] = tt;
            s_o[w] = om;
        }
        __syncthreads();
        if (w == 0) {
            ts = lane < ROW_CTA / 32 ? s_d[lane] : 0.0;
            tt = lane < ROW_CTA / 32 ? s_t[lane] : 0;
            om = lane < ROW_CTA / 32 ? s_o[lane] : 0;
            ts = warp_sum(ts);
            tt = warp_sum(tt);
            om = warp_sum(om);
            if (lane == 0) finish_node(u, b - a, ts, tt, om, f.sig1, f.sig2, f.Ccenter, f.t_own, f.o);
        }
        __syncthreads();
    }
}

int launch_finalize(const int32_t *rp, const int32_t *ci, const Scratch &s, int precision, int32_t n,
                    const ef_outputs &out, int num_sms, cudaStream_t st) {
    FinalArgs f{rp, ci, s.sig1, s.sig2, s.slotR, s.slotT, s.Ccenter, s.t_own, out};
    int64_t g = ((int64_t)n + 255) / 256;
    unsigned grid = (unsigned)(g < 1 ? 1 : (g > num_sms * 64 ? num_sms * 64 : g));
    if (precision == EF_PREC_FP64) {
        k_finalize<true><<<grid, 256, 0, st>>>(n, f);
        k_finalize_hub<true><<<num_sms * 4, ROW_CTA, 0, st>>>(n, s.bins, s.counters, f);
    } else {
        k_finalize<false><<<grid, 256, 0, st>>>(n, f);
        k_finalize_hub<false><<<num_sms * 4, ROW_CTA, 0, st>>>(n, s.bins, s.counters, f);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
