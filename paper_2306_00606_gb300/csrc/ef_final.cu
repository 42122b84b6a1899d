// Finalize pass of libef (Algorithm 1, Phase 3; Eq. 1).
//
// Per node v (one warp): sum the slots of v's row -- open-degree credits
// from every neighbour as middle node, triangle corrections and triangle
// counts found by neighbours as owners -- and add v's own middle-node credit
// and owned triangles.  Then
//   N_v = D(D-2) + sigma1,
//   S_v = D(D-1)(D-4) + 2(D-1) sigma1                      (v as middle)
//       + sigma2 - sigma1 + (D-4)(sigma1 - D) + omega - D^2 (v as an end)
//       - 8 t_v                                            (triangles)
// with D = D_v, sigma1 = sum of neighbour degrees, sigma2 = sum of their
// squares, omega = sum of the neighbours' sigma1 -- the exact integer sums of
// Algorithm 1's credited degrees, in closed form -- and
//   EF(v) = -sum over credited clusters of (d/S) ln(d/S) = ln S - T/S,
// with EF = 0 and flag = 1 when S = 0.
#include "ef_internal.cuh"

#include <type_traits>

namespace ef {

template <bool F64>
__global__ void __launch_bounds__(256) k_finalize(
    const int32_t *__restrict__ rp, int32_t n, const int32_t *__restrict__ D, const int64_t *__restrict__ sig1,
    const int64_t *__restrict__ sig2, const int64_t *__restrict__ omega, const void *__restrict__ slotR_,
    const double *__restrict__ slotC, const int32_t *__restrict__ slotT, const double *__restrict__ Ccenter,
    const double *__restrict__ tri_own, const int64_t *__restrict__ t_own, double *__restrict__ o_ef,
    int64_t *__restrict__ o_n, int64_t *__restrict__ o_s, double *__restrict__ o_t, int64_t *__restrict__ o_tri,
    uint8_t *__restrict__ o_flag) {
    using Acc = typename std::conditional<F64, double, float>::type;
    const Acc *slotR = reinterpret_cast<const Acc *>(slotR_);
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t vv = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); vv < n; vv += nwarps) {
        const int v = (int)vv;
        const int a = rp[v], b = rp[v + 1];
        double tr = 0.0, tc = 0.0;
        int64_t tt = 0;
        for (int e = a + lane; e < b; e += 32) {
            tr += (double)slotR[e];
            tc += slotC[e];
            tt += slotT[e];
        }
        tr = warp_sum(tr);
        tc = warp_sum(tc);
        tt = warp_sum(tt);
        if (lane == 0) {
            const int64_t d = b - a;
            const int64_t t = t_own[v] + tt;
            const double T = (d >= 2 ? Ccenter[v] : 0.0) + tr + 4.0 * (tri_own[v] + tc);
            const int64_t s1 = sig1[v], s2 = sig2[v], om = omega[v];
            const int64_t N = d * (d - 2) + s1;
            const int64_t S = d * (d - 1) * (d - 4) + 2 * (d - 1) * s1 + s2 - s1 + (d - 4) * (s1 - d) + om - d * d -
                              8 * t;
            double ef = 0.0;
            uint8_t fl = 1;
            if (S > 0) {
                const double Sd = (double)S;
                ef = log(Sd) - T / Sd;
                fl = 0;
            }
            if (o_ef) o_ef[v] = ef;
            if (o_n) o_n[v] = N;
            if (o_s) o_s[v] = S;
            if (o_t) o_t[v] = T;
            if (o_tri) o_tri[v] = t;
            if (o_flag) o_flag[v] = fl;
        }
    }
}

int launch_finalize(const int32_t *rp, const int32_t *ci, const Scratch &s, int precision, int32_t n,
                    const ef_outputs &out, cudaStream_t st) {
    (void)ci;
    int64_t g = ((int64_t)n + 7) / 8;
    unsigned grid = (unsigned)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
    if (precision == EF_PREC_FP64)
        k_finalize<true><<<grid, 256, 0, st>>>(rp, n, s.D, s.sig1, s.sig2, s.omega, s.slotR, s.slotC, s.slotT,
                                               s.Ccenter, s.tri_own, s.t_own, out.ef, out.n_clusters, out.s, out.t,
                                               out.triangles, out.flag);
    else
        k_finalize<false><<<grid, 256, 0, st>>>(rp, n, s.D, s.sig1, s.sig2, s.omega, s.slotR, s.slotC, s.slotT,
                                                s.Ccenter, s.tri_own, s.t_own, out.ef, out.n_clusters, out.s, out.t,
                                                out.triangles, out.flag);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
