// The learned ranking path, apart from the network itself:
// - node features;
// - a deterministic top-k selection on the device;
// - exact EF of chosen nodes (vertex-centric, Algorithm 1's credits
//   restricted to the chosen nodes).
//
// Exact EF of a chosen node v (T_v = middle + end + triangle parts, S_v and
// N_v in closed form as in the full pass):
// - middle and end: the wedge kernels of the full pass run with work bins
//   that hold only the chosen nodes and their neighbours (every middle node
//   whose clusters contain a chosen node), which gives Ccenter[v] and
//   Tacc[v] exactly, at the degree-class cost of those middle nodes;
// - triangles at v: per chosen node (k_nodes_final), each bringing the same
//   fixed-point correction 4 (f(s-6) - f(s-4)) as in the full pass.
// The chosen nodes of a ranking have the largest EF, which sit next to the
// hubs: their neighbourhoods cover most middle nodes (60-67% of the nodes of
// a BA graph for the top 1-2%), so this costs most of a wedge pass.
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

// The 16 features of every node (in the order of the oracle's FEATURE_NAMES).
// mode 1 uses the triangle counts tcnt, mode 0 takes t = 0.  BF16: each row
// standardised with the model's mean and standard deviation, z = (x - mean)
// * (1 / std) in FP32 as the network does it, and rounded to BF16, two
// features per word: exactly the network's first-layer operand, in 32 bytes
// per row instead of 64.
template <bool BF16>
__global__ void k_features(int32_t n, int mode, const int32_t *__restrict__ D, const int64_t *__restrict__ sig1,
                           const int64_t *__restrict__ sig2, const int64_t *__restrict__ omega,
                           const int32_t *__restrict__ nmin, const int32_t *__restrict__ nmax,
                           const int64_t *__restrict__ tcnt, float *__restrict__ X, const ModelDev *__restrict__ M) {
    __shared__ float s_mean[MLP_F], s_istd[MLP_F];
    if (BF16) {
        if (threadIdx.x < MLP_F) {
            s_mean[threadIdx.x] = M->mean[threadIdx.x];
            s_istd[threadIdx.x] = 1.0f / M->stdv[threadIdx.x];
        }
        __syncthreads();
    }
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
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
        if (BF16) {
            uint32_t wd[MLP_F / 2];
#pragma unroll
            for (int q = 0; q < MLP_F / 2; ++q)
                wd[q] = pack_bf16((f[2 * q] - s_mean[2 * q]) * s_istd[2 * q],
                                  (f[2 * q + 1] - s_mean[2 * q + 1]) * s_istd[2 * q + 1]);
            uint4 *dst = reinterpret_cast<uint4 *>(X) + (int64_t)v * 2;
            dst[0] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
            dst[1] = make_uint4(wd[4], wd[5], wd[6], wd[7]);
        } else {
            float4 *dst = reinterpret_cast<float4 *>(X + (int64_t)v * MLP_F);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
        }
    }
}

int launch_features(const Scratch &s, const RankScratch &r, int32_t n, int mode, const Tune &t, cudaStream_t st,
                    const ModelDev *std_model) {
    if (std_model)
        k_features<true><<<t.grid((int64_t)n, 256), 256, 0, st>>>(n, mode, s.D, s.sig1, s.sig2, s.omega, r.nbr_min,
                                                                 r.nbr_max, s.tcnt, r.x, std_model);
    else
        k_features<false><<<t.grid((int64_t)n, 256), 256, 0, st>>>(n, mode, s.D, s.sig1, s.sig2, s.omega, r.nbr_min,
                                                                  r.nbr_max, s.tcnt, r.x, nullptr);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ------------------------------------------------------------- top-k select
// The k largest of n keys (key 0 = not eligible), found digit by digit from
// the top (8-bit digits, histograms in shared memory, then one atomic per
// bin per block), then compacted in index order; among keys equal to the
// k-th largest the smallest indices are taken.  State in sel[]: 0 prefix,
// 1 still needed, 2 k.
__global__ void k_sel_init(uint64_t *sel, int64_t k) {
    sel[0] = 0;
    sel[1] = (uint64_t)k;
    sel[2] = (uint64_t)k;
}

__global__ void k_sel_hist(const uint64_t *__restrict__ key, int32_t n, const uint64_t *__restrict__ sel, int shift,
                           int32_t *__restrict__ hist) {
    __shared__ int32_t h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint64_t prefix = sel[0];
    const int hs = shift + 8;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint64_t kk = key[v];
        if (kk == 0) continue;
        if (hs < 64 && (kk >> hs) != (prefix >> hs)) continue;
        atomicAdd(&h[(kk >> shift) & 255], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, h[i]);
}

// 256 threads, thread i holding digit 255 - i: the digit d with (keys above
// d) < need <= (keys at or above d).
__global__ void __launch_bounds__(256) k_sel_pick(const int32_t *__restrict__ hist, uint64_t *sel, int shift) {
    __shared__ int64_t s_w[8];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int digit = 255 - tid;
    const int64_t mine = hist[digit];
    int64_t inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    int64_t before = 0;
    for (int i = 0; i < w; ++i) before += s_w[i];
    const int64_t above = before + inc - mine;   // keys in higher digits
    const int64_t need = (int64_t)sel[1];
    __syncthreads();
    if (above < need && above + mine >= need) {
        sel[0] |= (uint64_t)digit << shift;
        sel[1] = (uint64_t)(need - above);
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

// Selects the k largest keys of r.key (keys `bits` wide: 32 or 64) into
// r.list[0..k) (index order).  The caller guarantees 1 <= k <= number of
// nonzero keys.
int launch_select_top(const RankScratch &r, int32_t n, int64_t k, int bits, const Tune &t, cudaStream_t st) {
    const unsigned grid = t.grid((int64_t)n, 256);
    k_sel_init<<<1, 1, 0, st>>>(r.sel, k);
    for (int shift = bits - 8; shift >= 0; shift -= 8) {
        if (cudaMemsetAsync(r.hist, 0, 256 * sizeof(int32_t), st) != cudaSuccess) return -1;
        k_sel_hist<<<grid, 256, 0, st>>>(r.key, n, r.sel, shift, r.hist);
        k_sel_pick<<<1, 256, 0, st>>>(r.hist, r.sel, shift);
    }
    k_sel_ties<<<grid, 256, 0, st>>>(r.key, n, r.sel, r.flag);
    if (launch_scan(r.flag, r.pos, n, r.scan_tmp, st)) return -1;
    k_sel_flags<<<grid, 256, 0, st>>>(r.key, n, r.sel, r.pos, r.flag);
    if (launch_scan(r.flag, r.pos, n, r.scan_tmp, st)) return -1;
    k_scatter<<<grid, 256, 0, st>>>(r.flag, r.pos, n, r.list);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ------------------------------------------------------ exact EF of nodes
// mark[x] = 1 for every listed node and every neighbour of one: the middle
// nodes whose wedge credits reach a listed node.  Ids outside [0, n) set an
// error bit.
__global__ void k_mark_nbhd(const int32_t *__restrict__ list, int32_t k_max, const int32_t *__restrict__ kptr,
                            const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n,
                            int32_t *__restrict__ mark, int32_t *__restrict__ cnt) {
    const int k = kptr ? *kptr : k_max;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < k; i += nw) {   // a warp per listed node
        const int v = list[i];
        if (v < 0 || v >= n) {
            if (lane == 0) atomicOr(cnt + CNT_ERR, ERRB_NODE);
            continue;
        }
        if (lane == 0) mark[v] = 1;
        for (int e = rp[v] + lane; e < rp[v + 1]; e += 32) mark[ci[e]] = 1;
    }
}

// Work bins holding only the marked nodes (as middle nodes of the wedge
// kernels).  Counting per block in shared memory, one global atomic per bin
// per block, so the bins keep the node order within a block.
__global__ void k_bin_marked(const int32_t *__restrict__ mark, const int32_t *__restrict__ D, int32_t n, int hub_min,
                             int32_t *__restrict__ bins, int32_t *__restrict__ cnt) {
    __shared__ int s_cnt[NUM_BINS], s_base[NUM_BINS];
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        if (threadIdx.x < NUM_BINS) s_cnt[threadIdx.x] = 0;
        __syncthreads();
        const int v = (int)(base + threadIdx.x);
        int b0 = -1, b1 = -1, p0 = 0, p1 = 0;
        if (v < n && mark[v]) {
            const int d = D[v];
            if (d >= 1 && d <= SMALL_MAX) {
                b0 = d <= 4 ? BIN_S4 : d <= 8 ? BIN_S8 : d <= 16 ? BIN_S16 : BIN_S32;
            } else if (d > SMALL_MAX) {
                b0 = BIN_BIG;
                b1 = d < hub_min ? BIN_MID : BIN_HUB0 + max(0, min(31 - __clz(d) - 9, NUM_HUB_BUCKETS - 1));
            }
        }
        if (b0 >= 0) p0 = atomicAdd(&s_cnt[b0], 1);
        if (b1 >= 0) p1 = atomicAdd(&s_cnt[b1], 1);
        __syncthreads();
        if (threadIdx.x < NUM_BINS)
            s_base[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(cnt + threadIdx.x, s_cnt[threadIdx.x]) : 0;
        __syncthreads();
        if (b0 >= 0) bins[(size_t)b0 * n + s_base[b0] + p0] = v;
        if (b1 >= 0) bins[(size_t)b1 * n + s_base[b1] + p1] = v;
        __syncthreads();
    }
}

// mark: an n-int array free for this call (the row passes' out-degrees).
int launch_bin_nodes(const int32_t *list, int32_t k, const int32_t *kptr, const int32_t *rp, const int32_t *ci,
                     const Scratch &s, int32_t *mark, int32_t n, const Tune &t, cudaStream_t st) {
    if (cudaMemsetAsync(mark, 0, (size_t)n * sizeof(int32_t), st) != cudaSuccess) return -1;
    if (cudaMemsetAsync(s.counters, 0, NUM_BINS * sizeof(int32_t), st) != cudaSuccess) return -1;
    // the work counters of the big-node kernels (CNT_BIGITEM .. CNT_HUB; CNT_TRIFRAC stays)
    if (cudaMemsetAsync(s.counters + CNT_BIGITEM, 0, (CNT_HUB - CNT_BIGITEM + 1) * sizeof(int32_t), st) !=
        cudaSuccess)
        return -1;
    int64_t g = ((int64_t)k * 32 + 255) / 256;
    k_mark_nbhd<<<(unsigned)(g < 1 ? 1 : (g > 8192 ? 8192 : g)), 256, 0, st>>>(list, k, kptr, rp, ci, n, mark,
                                                                              s.counters);
    k_bin_marked<<<t.grid((int64_t)n, 256), 256, 0, st>>>(mark, s.D, n, t.hub_min, s.bins, s.counters);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Work bins of the marked nodes only (mark filled by the caller).
int launch_bin_marked(const int32_t *mark, const Scratch &s, int32_t n, const Tune &t, cudaStream_t st) {
    if (cudaMemsetAsync(s.counters, 0, NUM_BINS * sizeof(int32_t), st) != cudaSuccess) return -1;
    if (cudaMemsetAsync(s.counters + CNT_BIGITEM, 0, (CNT_HUB - CNT_BIGITEM + 1) * sizeof(int32_t), st) !=
        cudaSuccess)
        return -1;
    k_bin_marked<<<t.grid((int64_t)n, 256), 256, 0, st>>>(mark, s.D, n, t.hub_min, s.bins, s.counters);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

constexpr int NODE_THREADS = 256;
constexpr int NODE_ROW_SMEM = 4096;   // rows up to this length are staged for the triangle tests

// Is x adjacent to y?  Binary search in the shorter of the two sorted rows.
__device__ __forceinline__ bool adjacent(const int32_t *rp, const int32_t *ci, int x, int Dx, int y, int Dy) {
    const int a = Dx <= Dy ? x : y, b = Dx <= Dy ? y : x;
    const int s = rp[a], len = rp[a + 1] - s;
    const int p = lower_bound_i32(ci + s, len, b);
    return p < len && ci[s + p] == b;
}

// A CTA per listed node v: triangles at v and their corrections, then EF.
// T_v = Ccenter[v] (middle, open degrees) + Tacc[v] (end, open degrees, from
// the wedge pass over the marked middle nodes) + corrections.  Triangles are
// found either as adjacent pairs of N(v) (C(D_v, 2) tests in the shorter
// rows, each triangle once) or by streaming every neighbour's row against
// N(v) (sigma1(v) tests in a row held in shared memory, each triangle twice),
// whichever costs less.
template <bool F64>
__global__ void __launch_bounds__(NODE_THREADS) k_nodes_final(
    const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const int32_t *__restrict__ D,
    const int64_t *__restrict__ sig1, const int64_t *__restrict__ sig2, const int64_t *__restrict__ omega,
    const void *__restrict__ Ccenter, const double *__restrict__ Tacc, const int64_t *__restrict__ tq,
    const int32_t *__restrict__ cnt, const int32_t *__restrict__ list, int32_t k_max,
    const int32_t *__restrict__ kptr, int32_t n, const int64_t *__restrict__ qacc, const int64_t *__restrict__ tcnt,
    ef_outputs out) {
    __shared__ int32_t s_row[NODE_ROW_SMEM];
    __shared__ long long s_q[NODE_THREADS / 32], s_t[NODE_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int F = cnt[CNT_TRIFRAC];
    const int k = kptr ? *kptr : k_max;
    for (int i = blockIdx.x; i < k; i += gridDim.x) {
        const int v = list[i];
        if (v < 0 || v >= n) continue;   // reported by k_mark_nbhd (the whole CTA skips alike)
        const int a = rp[v], Dv = rp[v + 1] - a;
        const int64_t s1v = sig1[v];
        const bool global = qacc != nullptr;   // triangles already counted by the full pass
        const bool by_pairs = !global && (int64_t)Dv * (Dv - 1) / 2 * 16 <= s1v;
        const bool staged = !global && !by_pairs && Dv <= NODE_ROW_SMEM;
        if (staged)
            for (int e = threadIdx.x; e < Dv; e += NODE_THREADS) s_row[e] = ci[a + e];
        __syncthreads();
        int64_t q = 0, t = 0;   // by pairs: each triangle once; by streaming: twice
        if (global) {
        } else if (by_pairs) {
            for (int x = w; x < Dv; x += NODE_THREADS / 32) {
                const int bx = ci[a + x], Dx = D[bx];
                for (int y = x + 1 + lane; y < Dv; y += 32) {
                    const int by = ci[a + y], Dy = D[by];
                    if (adjacent(rp, ci, bx, Dx, by, Dy)) {
                        q += __ldg(tq + Dv + Dx + Dy);
                        ++t;
                    }
                }
            }
        } else {
            const int32_t *row = staged ? s_row : ci + a;
            for (int e = w; e < Dv; e += NODE_THREADS / 32) {
                const int u = row[e];
                const int ua = rp[u], Du = rp[u + 1] - ua;
                for (int jj = lane; jj < Du; jj += 32) {
                    const int x = ci[ua + jj];
                    if (x == v) continue;
                    const int p = lower_bound_i32(row, Dv, x);
                    if (p < Dv && row[p] == x) {
                        q += __ldg(tq + Dv + Du + D[x]);
                        ++t;
                    }
                }
            }
        }
        q = warp_sum(q);
        t = warp_sum(t);
        if (lane == 0) {
            s_q[w] = q;
            s_t[w] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t qs = 0, ts = 0;
            for (int j = 0; j < NODE_THREADS / 32; ++j) {
                qs += s_q[j];
                ts += s_t[j];
            }
            if (global) {
                qs = qacc[v];
                ts = tcnt[v];
            } else if (!by_pairs) {
                qs /= 2;   // each triangle was found through both of its other nodes
                ts /= 2;
            }
            const int64_t d = Dv, s2 = sig2[v], om = omega[v];
            const int64_t N = d * (d - 2) + s1v;
            const int64_t S =
                d * (d - 1) * (d - 4) + 2 * (d - 1) * s1v + s2 - s1v + (d - 4) * (s1v - d) + om - d * d - 8 * ts;
            const double cc = d >= 2 ? (double)reinterpret_cast<const AccT<F64> *>(Ccenter)[v] : 0.0;
            const double T = cc + Tacc[v] + ldexp((double)qs, -F);
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
            if (out.triangles) out.triangles[i] = ts;
            if (out.flag) out.flag[i] = fl;
        }
        __syncthreads();
    }
}

// With the full triangle pass done: a thread per listed node assembles T, S,
// N and EF from the accumulators (as the finalize pass does for all nodes).
template <bool F64>
__global__ void k_nodes_assemble(const int32_t *__restrict__ D, const int64_t *__restrict__ sig1,
                                 const int64_t *__restrict__ sig2, const int64_t *__restrict__ omega,
                                 const void *__restrict__ Ccenter, const double *__restrict__ Tacc,
                                 const int64_t *__restrict__ qacc, const int64_t *__restrict__ tcnt,
                                 const int32_t *__restrict__ cnt, const int32_t *__restrict__ list, int32_t k_max,
                                 const int32_t *__restrict__ kptr, int32_t n, ef_outputs out) {
    const int F = cnt[CNT_TRIFRAC];
    const int k = kptr ? *kptr : k_max;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const int v = list[i];
        if (v < 0 || v >= n) continue;   // reported by k_mark_nbhd
        const int64_t d = D[v], s1 = sig1[v], s2 = sig2[v], om = omega[v], t = tcnt[v];
        const int64_t N = d * (d - 2) + s1;
        const int64_t S = d * (d - 1) * (d - 4) + 2 * (d - 1) * s1 + s2 - s1 + (d - 4) * (s1 - d) + om - d * d - 8 * t;
        const double cc = d >= 2 ? (double)reinterpret_cast<const AccT<F64> *>(Ccenter)[v] : 0.0;
        const double T = cc + Tacc[v] + ldexp((double)qacc[v], -F);
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
}

// global_tri: take t and the corrections from the full triangle pass (qacc,
// tcnt) instead of counting per listed node.
int launch_nodes_exact(const int32_t *rp, const int32_t *ci, const Scratch &s, const int32_t *list, int32_t k,
                       const int32_t *kptr, int32_t n, int precision, bool global_tri, const ef_outputs &out,
                       const Tune &t, cudaStream_t st) {
    if (k <= 0) return 0;
    if (global_tri) {
        int64_t g = ((int64_t)k + 255) / 256;
        const unsigned ga = (unsigned)(g < 1 ? 1 : (g > (int64_t)t.num_sms * 16 ? (int64_t)t.num_sms * 16 : g));
        if (precision == EF_PREC_FP64)
            k_nodes_assemble<true><<<ga, 256, 0, st>>>(s.D, s.sig1, s.sig2, s.omega, s.Ccenter, s.Tacc, s.qacc, s.tcnt,
                                                       s.counters, list, k, kptr, n, out);
        else
            k_nodes_assemble<false><<<ga, 256, 0, st>>>(s.D, s.sig1, s.sig2, s.omega, s.Ccenter, s.Tacc, s.qacc,
                                                        s.tcnt, s.counters, list, k, kptr, n, out);
        return cudaGetLastError() == cudaSuccess ? 0 : -1;
    }
    const unsigned grid = (unsigned)(k < t.num_sms * 8 ? k : t.num_sms * 8);
    const int64_t *q = nullptr, *tc = nullptr;
    if (precision == EF_PREC_FP64)
        k_nodes_final<true><<<grid, NODE_THREADS, 0, st>>>(rp, ci, s.D, s.sig1, s.sig2, s.omega, s.Ccenter, s.Tacc,
                                                           s.tq, s.counters, list, k, kptr, n, q, tc, out);
    else
        k_nodes_final<false><<<grid, NODE_THREADS, 0, st>>>(rp, ci, s.D, s.sig1, s.sig2, s.omega, s.Ccenter,
                                                            s.Tacc, s.tq, s.counters, list, k, kptr, n, q, tc, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ------------------------------------------------------------ ranking glue
// Order-preserving 64-bit key of a finite double (never 0).
__device__ __forceinline__ uint64_t order_key(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Order-preserving 32-bit key of a finite float (never 0), in a 64-bit slot.
__device__ __forceinline__ uint64_t order_key32(float x) {
    const uint32_t b = __float_as_uint(x);
    return (uint64_t)((b >> 31) ? ~b : (b | 0x80000000u));
}

__global__ void k_keys_score(const float *__restrict__ score, int32_t n, uint64_t *__restrict__ key) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        key[v] = order_key32(score[v]);
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
