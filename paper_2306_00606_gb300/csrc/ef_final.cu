// Finalize pass of libef (Algorithm 1, Phase 3; Eq. 1).
//
// One thread per node v reads v's accumulators:
//   T_v = Ccenter[v]               (v as the middle node, open degrees)
//       + Tacc[v]                  (v as an end, open degrees)
//       + qacc[v] 2^-F             (triangle corrections, fixed point)
//   t_v = tcnt[v]
// and S_v and N_v, the exact integer sums of Algorithm 1's credited degrees
// and clusters, in closed form:
//   N_v = D(D-2) + sigma1,
//   S_v = D(D-1)(D-4) + 2(D-1) sigma1                      (v as middle)
//       + sigma2 - sigma1 + (D-4)(sigma1 - D) + omega - D^2 (v as an end)
//       - 8 t_v                                            (triangles)
// with D = D_v, sigma1 = sum of neighbour degrees, sigma2 = sum of their
// squares, omega = sum of the neighbours' sigma1.  Then
//   EF(v) = -sum over credited clusters of (d/S) ln(d/S) = ln S - T/S,
// with EF = 0 and flag = 1 when S = 0.  A node whose two symmetry
// fingerprints differ marks the input as asymmetric (a graph error).
//
// Precision: FP64 mode evaluates ln S - T/S in FP64.  FP32C evaluates it in
// FP32 (absolute error a few 1e-6) except at nodes of degree > HUB_FP64_DEG,
// where ln S is large and the cancellation in ln S - T/S is done in FP64.
#include "ef_internal.cuh"

namespace ef {

constexpr int HUB_FP64_DEG = 1000;

struct FinalArgs {
    const int32_t *D;
    const int64_t *sig1, *sig2, *omega;
    const uint64_t *fp_row, *fp_push;
    const double *Tacc;
    const void *Ccenter;
    const int64_t *qacc, *tcnt;
    int32_t *cnt;
    ef_outputs o;
};

template <bool F64>
__global__ void __launch_bounds__(256) k_finalize(int32_t n, FinalArgs f) {
    const int F = f.cnt[CNT_TRIFRAC];
    const double qscale = ldexp(1.0, -F);
    int err = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int64_t d = f.D[v];
        const int64_t t = f.tcnt[v];
        const int64_t s1 = f.sig1[v], s2 = f.sig2[v], om = f.omega[v];
        if (f.fp_row[v] != f.fp_push[v]) err |= ERRB_ASYM;
        const int64_t N = d * (d - 2) + s1;
        const int64_t S = d * (d - 1) * (d - 4) + 2 * (d - 1) * s1 + s2 - s1 + (d - 4) * (s1 - d) + om - d * d - 8 * t;
        const AccT<F64> cc = d >= 2 ? reinterpret_cast<const AccT<F64> *>(f.Ccenter)[v] : (AccT<F64>)0;
        const double T = ((double)cc + f.Tacc[v]) + (double)f.qacc[v] * qscale;
        double ef = 0.0;
        uint8_t fl = 1;
        if (S > 0) {
            fl = 0;
            if (F64 || d > HUB_FP64_DEG) {
                const double Sd = (double)S;
                ef = log(Sd) - T / Sd;
            } else {
                // ln S = ln(m) + e ln 2 with S = m 2^e, m in [0.5, 1).  ln 2 is split
                // into 45426/2^16 (16 significant bits, so e times it is exact) plus
                // the remainder ln 2 - 45426/2^16, keeping ln S at FP32 precision.
                int e2;
                const float Sf = (float)S;
                const float mant = frexpf(Sf, &e2);
                const float lnS = logf(mant) + (float)e2 * 0.693145751953125f + (float)e2 * 1.4286068203094e-06f;
                ef = (double)(lnS - __fdiv_rn((float)T, Sf));
            }
        }
        const ef_outputs &o = f.o;
        if (o.ef) o.ef[v] = ef;
        if (o.n_clusters) o.n_clusters[v] = N;
        if (o.s) o.s[v] = S;
        if (o.t) o.t[v] = T;
        if (o.triangles) o.triangles[v] = t;
        if (o.flag) o.flag[v] = fl;
    }
    err = __reduce_or_sync(FULL, err);
    if ((threadIdx.x & 31) == 0 && err) atomicOr(f.cnt + CNT_ERR, err);
}

int launch_finalize(const Scratch &s, int precision, int32_t n, const ef_outputs &out, const Tune &t,
                    cudaStream_t st) {
    const int num_sms = t.num_sms;
    const FinalArgs f{s.D,    s.sig1,    s.sig2, s.omega, s.fp_row,   s.fp_push,
                      s.Tacc, s.Ccenter, s.qacc, s.tcnt,  s.counters, out};
    int64_t g = ((int64_t)n + 255) / 256;
    unsigned grid = (unsigned)(g < 1 ? 1 : (g > (int64_t)num_sms * 32 ? (int64_t)num_sms * 32 : g));
    if (precision == EF_PREC_FP64) k_finalize<true><<<grid, 256, 0, st>>>(n, f);
    else k_finalize<false><<<grid, 256, 0, st>>>(n, f);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
