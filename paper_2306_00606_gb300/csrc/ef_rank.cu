// The learned ranking path, apart from the network itself:
// - node features;
// - a deterministic top-k selection on the device;
// - exact EF of chosen nodes (vertex-centric, Algorithm 1's credits
//   restricted to the chosen nodes).
//
// Exact EF of a chosen node v (T_v = middle + end + triangle parts, S_v and
// N_v in closed form as in the full pass):
// - middle: the wedge kernels run with work bins that hold only the chosen
//   nodes, which gives Ccenter[v] (the degree-class kernels for large D_v);
// - end: for every neighbour u and every j in N(u) other than v, one credit
//   of open degree D_u + D_v + D_j - 4; a CTA per chosen node streams N(u);
// - triangles: j in N(u) that is also in N(v) closes a triangle {v, u, j},
//   found twice (through u and through j); each triangle brings the same
//   fixed-point correction 4 (f(s-6) - f(s-4)) as in the full pass.
#include "ef_internal.cuh"

namespace ef {

// ------------------------------------------------------------------ features
// omega_v = sum over N(v) of sigma1(x); the smallest and largest neighbour
// degree.  Thread / warp / CTA per row as in the other row passes.
struct OmegaRow {
    int64_t om = 0;
    int mn = 0x7fffffff, mx = 0;
    __device__ __forceinline__ void add(int Dx, int64_t s1x) {
        om += s1x;
        mn = min(mn, Dx);
        mx = max(mx, Dx);
    }
};

__global__ void k_omega_mm(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n, int64_t m,
                           int tmax, int hub_min, const int32_t *__restrict__ D, const int64_t *__restrict__ sig1,
                           int64_t *__restrict__ omega, int32_t *__restrict__ nmin, int32_t *__restrict__ nmax) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n;
         base += nwarps * 32) {
        const int v = (int)(base + lane);
        const bool in = base + lane < n;
        const int a = in ? rp[v] : 0, b = in ? rp[v + 1] : 0;
        const bool ok = in && a >= 0 && a <= b && (int64_t)b <= m;
        const int Dv = ok ? b - a : 0;
        auto put = [&](int u, const OmegaRow &r) {
            omega[u] = r.om;
            if (nmin) {
                nmin[u] = r.mx ? r.mn : 0;
                nmax[u] = r.mx;
            }
        };
        if (in && Dv <= tmax) {
            OmegaRow r;
            for (int e0 = a; e0 < b; e0 += 4) {
                int x[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) x[q] = e0 + q < b ? ci[e0 + q] : -1;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (x[q] >= 0 && x[q] < n) r.add(D[x[q]], sig1[x[q]]);
            }
            put(v, r);
        }
        unsigned mid = __ballot_sync(FULL, Dv > tmax && Dv < hub_min);
        while (mid) {
            const int j = __ffs(mid) - 1;
            mid &= mid - 1;
            const int u = (int)(base + j);
            const int ua = __shfl_sync(FULL, a, j), ub = __shfl_sync(FULL, b, j);
            OmegaRow r;
            for (int e = ua + lane; e < ub; e += 32) {
                const int x = ci[e];
                if (x >= 0 && x < n) r.add(D[x], sig1[x]);
            }
            r.om = warp_sum(r.om);
            r.mn = __reduce_min_sync(FULL, r.mn);
            r.mx = __reduce_max_sync(FULL, r.mx);
            if (lane == 0) put(u, r);
        }
    }
}

__global__ void __launch_bounds__(ROW_CTA) k_omega_mm_hub(const int32_t *__restrict__ rp,
                                                          const int32_t *__restrict__ ci, int32_t n,
                                                          const int32_t *__restrict__ D,
                                                          const int64_t *__restrict__ sig1,
                                                          const int32_t *__restrict__ bins,
                                                          const int32_t *__restrict__ cnt, int64_t *__restrict__ omega,
                                                          int32_t *__restrict__ nmin, int32_t *__restrict__ nmax) {
    __shared__ int64_t s_om[ROW_CTA / 32];
    __shared__ int s_mn[ROW_CTA / 32], s_mx[ROW_CTA / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int total = hub_total(cnt);
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int u = hub_row(bins, n, cnt, it);
        const int a = rp[u], b = rp[u + 1];
        OmegaRow r;
        for (int e = a + threadIdx.x; e < b; e += ROW_CTA) {
            const int x = ci[e];
            if (x >= 0 && x < n) r.add(D[x], sig1[x]);
        }
        r.om = warp_sum(r.om);
        r.mn = __reduce_min_sync(FULL, r.mn);
        r.mx = __reduce_max_sync(FULL, r.mx);
        if (lane == 0) {
            s_om[w] = r.om;
            s_mn[w] = r.mn;
            s_mx[w] = r.mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            OmegaRow t;
            for (int i = 0; i < ROW_CTA / 32; ++i) {
                t.om += s_om[i];
                t.mn = min(t.mn, s_mn[i]);
                t.mx = max(t.mx, s_mx[i]);
            }
            omega[u] = t.om;
            if (nmin) {
                nmin[u] = t.mx ? t.mn : 0;
                nmax[u] = t.mx;
            }
        }
        __syncthreads();
    }
}

int launch_omega_mm(const int32_t *rp, const int32_t *ci, int32_t n, int64_t m, const Scratch &s,
                    const RankScratch &r, const Tune &t, cudaStream_t st) {
    k_omega_mm<<<t.grid((int64_t)n, 256), 256, 0, st>>>(rp, ci, n, m, t.row_thread_max, t.hub_min, s.D, s.sig1,
                                                         s.omega, r.nbr_min, r.nbr_max);
    k_omega_mm_hub<<<t.num_sms * 4, ROW_CTA, 0, st>>>(rp, ci, n, s.D, s.sig1, s.bins, s.counters, s.omega,
                                                      r.nbr_min, r.nbr_max);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// The 16 features of every node (in the order of the oracle's FEATURE_NAMES);
// also the symmetry check of the fingerprints.  mode 1 uses the triangle
// counts tcnt, mode 0 takes t = 0.
__global__ void k_features(int32_t n, int mode, const int32_t *__restrict__ D, const int64_t *__restrict__ sig1,
                           const int64_t *__restrict__ sig2, const int64_t *__restrict__ omega,
                           const int32_t *__restrict__ nmin, const int32_t *__restrict__ nmax,
                           const int64_t *__restrict__ tcnt, const uint64_t *__restrict__ fp_row,
                           const uint64_t *__restrict__ fp_push, float *__restrict__ X, int32_t *__restrict__ cnt) {
    int err = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (fp_row[v] != fp_push[v]) err |= ERRB_ASYM;
        const int64_t d = D[v], s1 = sig1[v], s2 = sig2[v], om = omega[v];
        const int64_t t = mode ? tcnt[v] : 0;
        const float fd = (float)d;
        const float mean = d > 0 ? (float)s1 / fd : 0.f;
        // d^2 var = d sigma2 - sigma1^2, formed in FP64 (no cancellation in FP32)
        const double vn = d > 0 ? fma((double)d, (double)s2, -(double)s1 * (double)s1) : 0.0;
        const float sd = d > 0 ? (float)sqrt(vn > 0.0 ? vn : 0.0) / fd : 0.f;
        const int64_t N = d * (d - 2) + s1;
        const int64_t So = d * (d - 1) * (d - 4) + 2 * (d - 1) * s1 + s2 - s1 + (d - 4) * (s1 - d) + om - d * d;
        const int64_t S = So - 8 * t;
        const int64_t pairs = d * (d - 1) / 2;
        float f[MLP_F];
        f[0] = log1pf(fd);
        f[1] = log1pf((float)s1);
        f[2] = log1pf((float)s2);
        f[3] = log1pf((float)om);
        f[4] = log1pf(mean);
        f[5] = log1pf(sd);
        f[6] = log1pf((float)nmin[v]);
        f[7] = log1pf((float)nmax[v]);
        f[8] = log1pf((float)N);
        f[9] = log1pf((float)So);
        f[10] = f[9] - f[8];
        f[11] = log1pf((float)t);
        f[12] = pairs > 0 ? (float)t / (float)pairs : 0.f;
        f[13] = log1pf((float)S);
        f[14] = f[2] - f[1];
        f[15] = f[3] - f[1];
        float4 *dst = reinterpret_cast<float4 *>(X + (int64_t)v * MLP_F);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
    }
    err = __reduce_or_sync(FULL, err);
    if ((threadIdx.x & 31) == 0 && err) atomicOr(cnt + CNT_ERR, err);
}

int launch_features(const Scratch &s, const RankScratch &r, int32_t n, int mode, const Tune &t, cudaStream_t st) {
    k_features<<<t.grid((int64_t)n, 256), 256, 0, st>>>(n, mode, s.D, s.sig1, s.sig2, s.omega, r.nbr_min, r.nbr_max,
                                                         s.tcnt, s.fp_row, s.fp_push, r.x, s.counters);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ------------------------------------------------------------- top-k select
// The k largest of n 64-bit keys (key 0 = not eligible), found digit by
// digit (four 16-bit passes), then compacted in index order; among keys
// equal to the k-th largest the smallest indices are taken.  State in
// sel[]: 0 prefix, 1 still needed, 2 k.
__global__ void k_sel_init(uint64_t *sel, int64_t k) {
    sel[0] = 0;
    sel[1] = (uint64_t)k;
    sel[2] = (uint64_t)k;
}

__global__ void k_sel_hist(const uint64_t *__restrict__ key, int32_t n, const uint64_t *__restrict__ sel, int shift,
                           int32_t *__restrict__ hist) {
    const uint64_t prefix = sel[0];
    const int hs = shift + 16;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint64_t kk = key[v];
        if (kk == 0) continue;
        if (hs < 64 && (kk >> hs) != (prefix >> hs)) continue;
        atomicAdd(hist + ((kk >> shift) & 0xffff), 1);
    }
}

// One CTA of 1024 threads: the digit d with (keys above d) < need <= (keys at
// or above d); thread 0 covers the highest 64 digits.
__global__ void __launch_bounds__(1024) k_sel_pick(const int32_t *__restrict__ hist, uint64_t *sel, int shift) {
    __shared__ int64_t s_w[33];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int hi = 65535 - 64 * tid;   // this thread's digits hi, hi-1, ..., hi-63
    int64_t mine = 0;
    for (int q = 0; q < 64; ++q) mine += hist[hi - q];
    int64_t inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t x = s_w[lane], xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, xi, o);
            if (lane >= o) xi += y;
        }
        s_w[lane] = xi - x;
    }
    __syncthreads();
    const int64_t above = s_w[w] + inc - mine;   // keys in higher digits than this thread's
    const int64_t need = (int64_t)sel[1];
    if (above < need && above + mine >= need) {
        int64_t acc = above;
        for (int q = 0; q < 64; ++q) {
            const int64_t h = hist[hi - q];
            if (acc + h >= need) {
                sel[0] |= (uint64_t)(hi - q) << shift;
                sel[1] = (uint64_t)(need - acc);
                break;
            }
            acc += h;
        }
    }
}

// flag[v] = 1 for keys equal to the threshold (first pass), then
// flag[v] = key above the threshold, or equal with tie rank < need.
__global__ void k_sel_ties(const uint64_t *__restrict__ key, int32_t n, const uint64_t *__restrict__ sel,
                           int32_t *__restrict__ flag) {
    const uint64_t T = sel[0];
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        flag[v] = key[v] != 0 && key[v] == T;
}

__global__ void k_sel_flags(const uint64_t *__restrict__ key, int32_t n, const uint64_t *__restrict__ sel,
                            const int32_t *__restrict__ tie_pos, int32_t *__restrict__ flag) {
    const uint64_t T = sel[0];
    const int64_t need = (int64_t)sel[1];
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint64_t kk = key[v];
        flag[v] = kk != 0 && (kk > T || (kk == T && tie_pos[v] < need));
    }
}

__global__ void k_scatter(const int32_t *__restrict__ flag, const int32_t *__restrict__ pos, int32_t n,
                          int32_t *__restrict__ list) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (flag[v]) list[pos[v]] = v;
}

// Selects the k largest keys of r.key into r.list[0..k) (index order).  The
// caller guarantees 1 <= k <= number of nonzero keys.
int launch_select_top(const RankScratch &r, int32_t n, int64_t k, const Tune &t, cudaStream_t st) {
    const unsigned grid = t.grid((int64_t)n, 256);
    k_sel_init<<<1, 1, 0, st>>>(r.sel, k);
    for (int shift = 48; shift >= 0; shift -= 16) {
        if (cudaMemsetAsync(r.hist, 0, 65536 * sizeof(int32_t), st) != cudaSuccess) return -1;
        k_sel_hist<<<grid, 256, 0, st>>>(r.key, n, r.sel, shift, r.hist);
        k_sel_pick<<<1, 1024, 0, st>>>(r.hist, r.sel, shift);
    }
    k_sel_ties<<<grid, 256, 0, st>>>(r.key, n, r.sel, r.flag);
    if (launch_scan(r.flag, r.pos, n, r.scan_tmp, st)) return -1;
    k_sel_flags<<<grid, 256, 0, st>>>(r.key, n, r.sel, r.pos, r.flag);
    if (launch_scan(r.flag, r.pos, n, r.scan_tmp, st)) return -1;
    k_scatter<<<grid, 256, 0, st>>>(r.flag, r.pos, n, r.list);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ------------------------------------------------------ exact EF of nodes
// Work bins holding only the listed nodes (as middle nodes of the wedge
// kernels); node ids outside [0, n) set an error bit.
__global__ void k_bin_nodes(const int32_t *__restrict__ list, int32_t k_max, const int32_t *__restrict__ kptr,
                            const int32_t *__restrict__ D, int32_t n, int hub_min, int32_t *__restrict__ bins,
                            int32_t *__restrict__ cnt) {
    const int k = kptr ? *kptr : k_max;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const int v = list[i];
        if (v < 0 || v >= n) {
            atomicOr(cnt + CNT_ERR, ERRB_NODE);
            continue;
        }
        const int d = D[v];
        int b0 = -1, b1 = -1;
        if (d >= 1 && d <= SMALL_MAX) {
            b0 = d <= 4 ? BIN_S4 : d <= 8 ? BIN_S8 : d <= 16 ? BIN_S16 : BIN_S32;
        } else if (d > SMALL_MAX) {
            b0 = BIN_BIG;
            b1 = d < hub_min ? BIN_MID : BIN_HUB0 + max(0, min(31 - __clz(d) - 9, NUM_HUB_BUCKETS - 1));
        }
        if (b0 >= 0) bins[(size_t)b0 * n + atomicAdd(cnt + b0, 1)] = v;
        if (b1 >= 0) bins[(size_t)b1 * n + atomicAdd(cnt + b1, 1)] = v;
    }
}

int launch_bin_nodes(const int32_t *list, int32_t k, const int32_t *kptr, const Scratch &s, int32_t n, int hub_min,
                     cudaStream_t st) {
    if (cudaMemsetAsync(s.counters, 0, NUM_BINS * sizeof(int32_t), st) != cudaSuccess) return -1;
    // the work counters of the big-node kernels (CNT_BIGITEM .. CNT_HUB; CNT_TRIFRAC stays)
    if (cudaMemsetAsync(s.counters + CNT_BIGITEM, 0, (CNT_HUB - CNT_BIGITEM + 1) * sizeof(int32_t), st) !=
        cudaSuccess)
        return -1;
    int64_t g = ((int64_t)k + 255) / 256;
    k_bin_nodes<<<(unsigned)(g < 1 ? 1 : (g > 4096 ? 4096 : g)), 256, 0, st>>>(list, k, kptr, s.D, n, hub_min,
                                                                              s.bins, s.counters);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

constexpr int NODE_THREADS = 256;
constexpr int NODE_ROW_SMEM = 4096;   // rows up to this length are staged for the triangle tests

template <bool F64>
__global__ void __launch_bounds__(NODE_THREADS) k_nodes_exact(
    const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const int32_t *__restrict__ D,
    const int64_t *__restrict__ sig1, const int64_t *__restrict__ sig2, const int64_t *__restrict__ omega,
    const void *__restrict__ Ccenter, const double *__restrict__ ftab, const int64_t *__restrict__ tq,
    const int32_t *__restrict__ cnt, const int32_t *__restrict__ list, int32_t k_max,
    const int32_t *__restrict__ kptr, int32_t n, ef_outputs out) {
    __shared__ int32_t s_row[NODE_ROW_SMEM];
    __shared__ double s_acc[NODE_THREADS / 32];
    __shared__ long long s_q[NODE_THREADS / 32], s_t[NODE_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int F = cnt[CNT_TRIFRAC];
    const int k = kptr ? *kptr : k_max;
    for (int i = blockIdx.x; i < k; i += gridDim.x) {
        const int v = list[i];
        if (v < 0 || v >= n) continue;   // reported by k_bin_nodes (the whole CTA skips alike)
        const int a = rp[v], Dv = rp[v + 1] - a;
        const bool staged = Dv <= NODE_ROW_SMEM;
        if (staged)
            for (int e = threadIdx.x; e < Dv; e += NODE_THREADS) s_row[e] = ci[a + e];
        __syncthreads();
        const int32_t *row = staged ? s_row : ci + a;
        SumAcc<AccT<F64>> acc;
        int64_t q2 = 0, t2 = 0;
        for (int e = w; e < Dv; e += NODE_THREADS / 32) {
            const int u = row[e];
            const int ua = rp[u], Du = rp[u + 1] - ua;
            const int base = Du + Dv - 4;
            for (int jj = lane; jj < Du; jj += 32) {
                const int x = ci[ua + jj];
                if (x == v) continue;
                const int Dx = D[x];
                if constexpr (F64) acc.add(__ldg(ftab + base + Dx));
                else acc.add(dlog2d((float)(base + Dx)));
                const int p = lower_bound_i32(row, Dv, x);
                if (p < Dv && row[p] == x) {
                    q2 += __ldg(tq + Dv + Du + Dx);
                    ++t2;
                }
            }
        }
        double end = F64 ? (double)acc.get() : (double)acc.get() * LN2;
        end = warp_sum(end);
        q2 = warp_sum(q2);
        t2 = warp_sum(t2);
        if (lane == 0) {
            s_acc[w] = end;
            s_q[w] = q2;
            s_t[w] = t2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double e_sum = 0.0;
            int64_t qs = 0, ts = 0;
            for (int q = 0; q < NODE_THREADS / 32; ++q) {
                e_sum += s_acc[q];
                qs += s_q[q];
                ts += s_t[q];
            }
            const int64_t d = Dv, t = ts / 2, s1 = sig1[v], s2 = sig2[v], om = omega[v];
            const int64_t N = d * (d - 2) + s1;
            const int64_t S =
                d * (d - 1) * (d - 4) + 2 * (d - 1) * s1 + s2 - s1 + (d - 4) * (s1 - d) + om - d * d - 8 * t;
            const double cc = d >= 2 ? (double)reinterpret_cast<const AccT<F64> *>(Ccenter)[v] : 0.0;
            const double T = cc + e_sum + ldexp((double)(qs / 2), -F);
            double ef = 0.0;
            uint8_t fl = 1;
            if (S > 0) {
                ef = log((double)S) - T / (double)S;
                fl = 0;
            }
            if (out.ef) out.ef[i] = ef;
            if (out.n_clusters) out.n_clusters[i] = N;
            if (out.s) out.s[i] = S;
            if (out.t) out.t[i] = T;
            if (out.triangles) out.triangles[i] = t;
            if (out.flag) out.flag[i] = fl;
        }
        __syncthreads();
    }
}

int launch_nodes_exact(const int32_t *rp, const int32_t *ci, const Scratch &s, const int32_t *list, int32_t k,
                       const int32_t *kptr, int32_t n, int precision, const ef_outputs &out, const Tune &t,
                       cudaStream_t st) {
    if (k <= 0) return 0;
    const unsigned grid = (unsigned)(k < t.num_sms * 8 ? k : t.num_sms * 8);
    if (precision == EF_PREC_FP64)
        k_nodes_exact<true><<<grid, NODE_THREADS, 0, st>>>(rp, ci, s.D, s.sig1, s.sig2, s.omega, s.Ccenter, s.ftab,
                                                           s.tq, s.counters, list, k, kptr, n, out);
    else
        k_nodes_exact<false><<<grid, NODE_THREADS, 0, st>>>(rp, ci, s.D, s.sig1, s.sig2, s.omega, s.Ccenter,
                                                            s.ftab, s.tq, s.counters, list, k, kptr, n, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ------------------------------------------------------------ ranking glue
// Order-preserving 64-bit key of a finite double (never 0).
__device__ __forceinline__ uint64_t order_key(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_keys_score(const float *__restrict__ score, int32_t n, uint64_t *__restrict__ key) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        key[v] = order_key((double)score[v]);
}

// role[v]: bit 1 candidate (from the selected list), bit 2 audit (node v is
// sampled when splitmix64(seed, v) < threshold).
__global__ void k_roles(const int32_t *__restrict__ cand, int32_t kc, int32_t n, uint64_t seed, uint64_t threshold,
                        int32_t *__restrict__ role) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * ((uint64_t)(uint32_t)v + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        role[v] = z < threshold ? 2 : 0;
    }
}

__global__ void k_mark(const int32_t *__restrict__ list, int32_t k, int bit, int32_t *__restrict__ role) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) role[list[i]] |= bit;
}

__global__ void k_flag_role(const int32_t *__restrict__ role, int32_t n, int mask, int32_t *__restrict__ flag) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        flag[v] = (role[v] & mask) != 0;
}

// exact EF by list position -> per node, and the keys of the candidates
__global__ void k_exact_keys(const int32_t *__restrict__ L, const int32_t *__restrict__ kL,
                             const double *__restrict__ exact, const int32_t *__restrict__ role,
                             double *__restrict__ exact_node, uint64_t *__restrict__ key) {
    const int k = *kL;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const int v = L[i];
        exact_node[v] = exact[i];
        if (role[v] & 1) key[v] = order_key(exact[i]);
    }
}

__global__ void k_gather_top(const int32_t *__restrict__ list, int32_t k, const double *__restrict__ exact_node,
                             int32_t *__restrict__ out_idx, double *__restrict__ out_ef) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const int v = list[i];
        if (out_idx) out_idx[i] = v;
        if (out_ef) out_ef[i] = exact_node[v];
    }
}

__global__ void k_gather_audit(const int32_t *__restrict__ list, const int32_t *__restrict__ ka,
                               const float *__restrict__ score, const double *__restrict__ exact_node,
                               float *__restrict__ a_score, double *__restrict__ a_exact) {
    const int k = *ka;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const int v = list[i];
        a_score[i] = score[v];
        a_exact[i] = exact_node[v];
    }
}

static inline unsigned grid_n(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (unsigned)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

int launch_keys_score(const float *score, int32_t n, uint64_t *key, cudaStream_t st) {
    k_keys_score<<<grid_n(n), 256, 0, st>>>(score, n, key);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_roles(const int32_t *cand, int32_t kc, int32_t n, uint64_t seed, uint64_t threshold, int32_t *role,
                 cudaStream_t st) {
    k_roles<<<grid_n(n), 256, 0, st>>>(cand, kc, n, seed, threshold, role);
    k_mark<<<grid_n(kc), 256, 0, st>>>(cand, kc, 1, role);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Compact the nodes with (role & mask) into list (node order); the count
// lands in pos[n].
int launch_compact_role(const int32_t *role, int32_t n, int mask, int32_t *flag, int32_t *pos, int32_t *tmp,
                        int32_t *list, cudaStream_t st) {
    k_flag_role<<<grid_n(n), 256, 0, st>>>(role, n, mask, flag);
    if (launch_scan(flag, pos, n, tmp, st)) return -1;
    k_scatter<<<grid_n(n), 256, 0, st>>>(flag, pos, n, list);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_exact_keys(const int32_t *L, const int32_t *kL, int32_t kmax, const double *exact, const int32_t *role,
                      double *exact_node, uint64_t *key, cudaStream_t st) {
    k_exact_keys<<<grid_n(kmax), 256, 0, st>>>(L, kL, exact, role, exact_node, key);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_gather_top(const int32_t *list, int32_t k, const double *exact_node, int32_t *out_idx, double *out_ef,
                      cudaStream_t st) {
    k_gather_top<<<grid_n(k), 256, 0, st>>>(list, k, exact_node, out_idx, out_ef);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_gather_audit(const int32_t *list, const int32_t *ka, int32_t kmax, const float *score,
                        const double *exact_node, float *a_score, double *a_exact, cudaStream_t st) {
    k_gather_audit<<<grid_n(kmax), 256, 0, st>>>(list, ka, score, exact_node, a_score, a_exact);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
