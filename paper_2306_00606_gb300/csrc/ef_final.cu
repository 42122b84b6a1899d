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
// with EF = 0 and flag = 1 when S = 0.
//
// Precision: FP64 mode evaluates ln S - T/S in FP64 (ln_ge1, div_by, both
// within about 1e-14 relative).  FP32C evaluates it in
// FP32 (absolute error a few 1e-6) except at nodes of degree > HUB_FP64_DEG,
// where ln S is large and the cancellation in ln S - T/S is done in FP64.
//
// A sharded computation ends in k_finalize_sums: the shards' summed
// partials already hold N and the open-degree sum S + 8t of every node, so
// it needs no pass over the graph.  Its FP32C test for FP64 evaluation is on
// S instead of the degree: S >= D (D-1) (D-4) (v's own clusters as middle
// node have degree >= D - 4), so S > HUB_FP64_S holds at every node of
// degree > HUB_FP64_DEG.
#include "ef_internal.cuh"

#include <mutex>

namespace ef {

constexpr int HUB_FP64_DEG = 1000;
constexpr int64_t HUB_FP64_S = (int64_t)HUB_FP64_DEG * (HUB_FP64_DEG - 1) * (HUB_FP64_DEG - 4);

// ln x for x >= 1 in FP64 with a dozen FP64 instructions (this GPU runs FP64
// at a thirty-second of the FP32 rate): x = m 2^e with m in [1, 2); the top
// eight bits of m pick c_k = 1 + (k + 1/2)/256, whose ln and reciprocal come
// from a table (g_lnc, g_rcc, computed once per device with the library
// log); r = m / c_k - 1 lies within 2^-9, and ln(1 + r) = r - r^2/2 + r^3/3
// - r^4/4 leaves out less than |r|^5/5 < 6e-15.  A numpy emulation over
// 3e5 values of S in [1, 2^62] gave errors below 1.5e-14.
__device__ double g_lnc[256], g_rcc[256];

__global__ void k_init_lnc() {
    const int k = threadIdx.x;
    const double c = 1.0 + ((double)k + 0.5) / 256.0;
    g_lnc[k] = log(c);
    g_rcc[k] = 1.0 / c;
}

__device__ __forceinline__ double ln_ge1(double x) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    const int k = (int)((b >> 44) & 0xff);
    const double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    const double r = fma(m, g_rcc[k], -1.0);
    const double p = r * fma(r, fma(r, fma(r, -0.25, 1.0 / 3.0), -0.5), 1.0);
    return fma((double)e, LN2, g_lnc[k] + p);
}

// T / S in FP64: an FP32 reciprocal (22 bits) refined by one Newton step
// (44 bits), then one product.
__device__ __forceinline__ double div_by(double T, double Sd) {
    const double y0 = (double)__frcp_rn((float)Sd);
    const double y1 = fma(y0, fma(-Sd, y0, 1.0), y0);
    return T * y1;
}

// EF = ln S - T / S for S > 0; wide: in FP64 also in FP32C mode.
template <bool F64>
__device__ __forceinline__ double ef_value(int64_t S, double T, bool wide) {
    if (F64 || wide) {
        const double Sd = (double)S;
        return ln_ge1(Sd) - div_by(T, Sd);
    }
    // ln S = ln(m) + e ln 2 with S = m 2^e, m in [0.5, 1).  ln 2 is split
    // into 45426/2^16 (16 significant bits, so e times it is exact) plus
    // the remainder ln 2 - 45426/2^16, keeping ln S at FP32 precision.
    int e2;
    const float Sf = (float)S;
    const float mant = frexpf(Sf, &e2);
    const float lnS = logf(mant) + (float)e2 * 0.693145751953125f + (float)e2 * 1.4286068203094e-06f;
    return (double)(lnS - __fdiv_rn((float)T, Sf));
}

struct FinalArgs {
    const int32_t *D;
    const int64_t *sig1, *sig2, *omega;
    const double *Tacc;
    const void *Ccenter;
    const int64_t *qacc, *tcnt;
    int32_t *cnt;
    ef_outputs o;
};

template <bool F64>
__global__ void __launch_bounds__(256) k_finalize(int32_t n, FinalArgs f) {
    if (gate_closed(f.cnt)) return;
    const int F = f.cnt[CNT_TRIFRAC];
    const double qscale = ldexp(1.0, -F);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int64_t d = f.D[v];
        const int64_t t = f.tcnt[v];
        const int64_t s1 = f.sig1[v], s2 = f.sig2[v], om = f.omega[v];
        const int64_t N = d * (d - 2) + s1;
        const int64_t S = d * (d - 1) * (d - 4) + 2 * (d - 1) * s1 + s2 - s1 + (d - 4) * (s1 - d) + om - d * d - 8 * t;
        const AccT<F64> cc = d >= 2 ? reinterpret_cast<const AccT<F64> *>(f.Ccenter)[v] : (AccT<F64>)0;
        const double T = ((double)cc + f.Tacc[v]) + (double)f.qacc[v] * qscale;
        double ef = 0.0;
        uint8_t fl = 1;
        if (S > 0) {
            fl = 0;
            ef = ef_value<F64>(S, T, d > HUB_FP64_DEG);
        }
        const ef_outputs &o = f.o;
        if (o.ef) o.ef[v] = ef;
        if (o.n_clusters) o.n_clusters[v] = N;
        if (o.s) o.s[v] = S;
        if (o.t) o.t[v] = T;
        if (o.triangles) o.triangles[v] = t;
        if (o.flag) o.flag[v] = fl;
    }
}

// From the shards' summed partials: T_v = t + q 2^-F, S_v = S_open - 8 t_v.
template <bool F64>
__global__ void __launch_bounds__(256) k_finalize_sums(int32_t n, ef_partials p, int32_t frac, ef_outputs o) {
    const double qscale = ldexp(1.0, -frac);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int64_t t = p.triangles[v];
        const int64_t S = p.s_open[v] - 8 * t;
        const double T = p.t[v] + (double)p.q[v] * qscale;
        double ef = 0.0;
        uint8_t fl = 1;
        if (S > 0) {
            fl = 0;
            ef = ef_value<F64>(S, T, S > HUB_FP64_S);
        }
        if (o.ef) o.ef[v] = ef;
        if (o.n_clusters) o.n_clusters[v] = p.n_clusters[v];
        if (o.s) o.s[v] = S;
        if (o.t) o.t[v] = T;
        if (o.triangles) o.triangles[v] = t;
        if (o.flag) o.flag[v] = fl;
    }
}

// The ln table of ln_ge1 on the current device, once (before any capture).
int prepare_final_tables() {
    static std::mutex mu;
    static bool ready[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
    std::lock_guard<std::mutex> lk(mu);
    if (ready[dev]) return 0;
    k_init_lnc<<<1, 256>>>();
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess) return -1;
    ready[dev] = true;
    return 0;
}

static inline unsigned grid_n(int32_t n, const Tune &t) {
    int64_t g = ((int64_t)n + 255) / 256;
    const int64_t cap = (int64_t)t.num_sms * 32;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

int launch_finalize(const Scratch &s, int precision, int32_t n, const ef_outputs &out, const Tune &t,
                    cudaStream_t st) {
    const FinalArgs f{s.D, s.sig1, s.sig2, s.omega, s.Tacc, s.Ccenter, s.qacc, s.tcnt, s.counters, out};
    if (precision == EF_PREC_FP64) k_finalize<true><<<grid_n(n, t), 256, 0, st>>>(n, f);
    else k_finalize<false><<<grid_n(n, t), 256, 0, st>>>(n, f);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_finalize_sums(const ef_partials &p, int precision, int32_t n, int32_t frac_bits, const ef_outputs &out,
                         const Tune &t, cudaStream_t st) {
    if (precision == EF_PREC_FP64) k_finalize_sums<true><<<grid_n(n, t), 256, 0, st>>>(n, p, frac_bits, out);
    else k_finalize_sums<false><<<grid_n(n, t), 256, 0, st>>>(n, p, frac_bits, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
