// Preparation passes of libef: CSR validation, degrees, neighbour-degree sums,
// work binning, degree orientation for triangle listing, reverse slots, the
// f(d) = d ln d table, and a device-wide exclusive scan.
//
// Algorithm 1's Phase 2 needs |Adj(x)| of every cluster member; the degree
// array D is the only per-node quantity the wedge pass reads besides the CSR.
#include "ef_internal.cuh"

namespace ef {

// ------------------------------------------------------------------ degrees
__global__ void k_degrees(const int32_t *__restrict__ rp, int32_t n, int64_t m, int32_t *__restrict__ D,
                          int32_t *__restrict__ cnt) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    int mx = 0, err = 0;
    if (v < n) {
        int a = rp[v], b = rp[v + 1];
        if (a < 0 || b < a || (int64_t)b > m) {
            err |= ERRB_ROWPTR;
            D[v] = 0;
        } else {
            D[v] = b - a;
            mx = b - a;
        }
    }
    if (v == 0 && (rp[0] != 0 || (int64_t)rp[n] != m)) err |= ERRB_ROWPTR;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(FULL, mx, o));
        err |= __shfl_xor_sync(FULL, err, o);
    }
    __shared__ int s_mx[32], s_err[32];
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { s_mx[w] = mx; s_err[w] = err; }
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        mx = l < nw ? s_mx[l] : 0;
        err = l < nw ? s_err[l] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mx = max(mx, __shfl_xor_sync(FULL, mx, o));
            err |= __shfl_xor_sync(FULL, err, o);
        }
        if (l == 0) {
            if (mx) atomicMax(cnt + CNT_MAXDEG, mx);
            if (err) atomicOr(cnt + CNT_ERR, err);
        }
    }
}

// ------------------------------------------- per-row checks and neighbour sums
// One warp per row: range, self-loop and strict-order checks; sigma1, sigma2
// and the out-degree of v in the (degree, id) order.
__global__ void k_row_stats(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n, int64_t m,
                            const int32_t *__restrict__ D, int64_t *__restrict__ sig1, int64_t *__restrict__ sig2,
                            int32_t *__restrict__ outdeg, int32_t *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t v = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n; v += nwarps) {
        int a = rp[v], b = rp[v + 1];
        bool ok = a >= 0 && a <= b && (int64_t)b <= m;
        int Dv = ok ? b - a : 0;
        int64_t s1 = 0, s2 = 0;
        int od = 0, err = 0;
        if (ok) {
            for (int e = a + lane; e < b; e += 32) {
                int x = ci[e];
                if (x < 0 || x >= n) { err |= ERRB_RANGE; continue; }
                if (x == (int)v) err |= ERRB_SELFLOOP;
                if (e > a && ci[e - 1] >= x) err |= ERRB_UNSORTED;
                int Dx = D[x];
                s1 += Dx;
                s2 += (int64_t)Dx * Dx;
                od += rank_less(Dv, (int)v, Dx, x) ? 1 : 0;
            }
        }
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        od = warp_sum(od);
        err = __reduce_or_sync(FULL, err);
        if (lane == 0) {
            sig1[v] = s1;
            sig2[v] = s2;
            outdeg[v] = od;
            if (err) atomicOr(cnt + CNT_ERR, err);
        }
    }
}

// ------------------------------------------------------------------- binning
__global__ void k_bin(const int32_t *__restrict__ D, const int32_t *__restrict__ outdeg, int32_t n,
                      int32_t *__restrict__ bins, int32_t *__restrict__ cnt) {
    __shared__ int s_cnt[NUM_BINS], s_base[NUM_BINS];
    if (threadIdx.x < NUM_BINS) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    int wb = -1, tb = -1, pw = 0, pt = 0;
    if (v < n) {
        int d = D[v];
        if (d >= 1) wb = d <= 4 ? BIN_S4 : d <= 8 ? BIN_S8 : d <= 16 ? BIN_S16 : d <= SMALL_MAX ? BIN_S32 : BIN_BIG;
        int o = outdeg[v];
        if (o >= 2) tb = o <= TRI_WARP_CAP ? BIN_TW : BIN_TC;
    }
    if (wb >= 0) pw = atomicAdd(&s_cnt[wb], 1);
    if (tb >= 0) pt = atomicAdd(&s_cnt[tb], 1);
    __syncthreads();
    if (threadIdx.x < NUM_BINS) s_base[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(cnt + threadIdx.x, s_cnt[threadIdx.x]) : 0;
    __syncthreads();
    if (wb >= 0) bins[(size_t)wb * n + s_base[wb] + pw] = v;
    if (tb >= 0) bins[(size_t)tb * n + s_base[tb] + pt] = v;
}

// ------------------------------------------- reverse slots and orientation
// One warp per row u.  For each slot e = (u -> x): rev[e] = position of u in
// N(x) (binary search; missing -> asymmetric input); omega[u] = sum of
// sigma1 over N(u); and the out-neighbours x of u in (degree, id) order are
// appended to the oriented CSR in ascending id order, with D_x and rev[e].
__global__ void k_rev_fill(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n, int64_t m,
                           const int32_t *__restrict__ D, const int64_t *__restrict__ sig1,
                           const int32_t *__restrict__ out_ptr, int32_t *__restrict__ rev,
                           int32_t *__restrict__ out_col, int32_t *__restrict__ out_D,
                           int32_t *__restrict__ out_rslot, int64_t *__restrict__ omega,
                           int32_t *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t vv = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); vv < n; vv += nwarps) {
        const int v = (int)vv;
        const int a = rp[v], b = rp[v + 1];
        // rows and columns that failed validation are skipped (memory safety
        // only: the call returns EF_ERR_GRAPH before any later pass runs)
        const bool ok = a >= 0 && a <= b && (int64_t)b <= m;
        const int Dv = ok ? b - a : 0;
        int base = out_ptr[v];
        int64_t om = 0;
        int err = 0;
        for (int e0 = a; ok && e0 < b; e0 += 32) {
            int e = e0 + lane;
            bool act = e < b;
            int x = act ? ci[e] : 0;
            bool xin = act && x >= 0 && x < n;
            int Dx = xin ? D[x] : 0;
            int p = e;
            if (act) {
                int xa = xin ? rp[x] : 0, xb = xin ? rp[x + 1] : 0;
                if (xin && xa >= 0 && xa <= xb && (int64_t)xb <= m) {
                    int pos = xa + lower_bound_i32(ci + xa, xb - xa, v);
                    if (pos < xb && ci[pos] == v) p = pos;
                    else err |= ERRB_ASYM;
                    om += sig1[x];
                } else {
                    err |= ERRB_ASYM;
                }
                rev[e] = p;
            }
            bool isout = xin && rank_less(Dv, v, Dx, x);
            unsigned bal = __ballot_sync(FULL, isout);
            if (isout) {
                int k = base + __popc(bal & ((1u << lane) - 1u));
                out_col[k] = x;
                out_D[k] = Dx;
                out_rslot[k] = p;
            }
            base += __popc(bal);
        }
        om = warp_sum(om);
        err = __reduce_or_sync(FULL, err);
        if (lane == 0) {
            omega[v] = om;
            if (err) atomicOr(cnt + CNT_ERR, err);
        }
    }
}

// Work items of the big middle nodes: ceil(D / BIG_ROWS) each; entries past
// the bin count are 0 so a scan over n gives the item offsets.
__global__ void k_big_chunks(const int32_t *__restrict__ D, const int32_t *__restrict__ big_list,
                             const int32_t *__restrict__ cnt, int32_t n, int32_t *__restrict__ chunks) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int nb = cnt[BIN_BIG];
    chunks[i] = i < nb ? (D[big_list[i]] + BIG_ROWS - 1) / BIG_ROWS : 0;
}

// -------------------------------------------------------------- f(d) table
__global__ void k_ftab(double *__restrict__ ftab, const int32_t *__restrict__ maxdeg, int64_t cap) {
    int64_t L = 3 * (int64_t)(*maxdeg) + 1;
    if (L > cap) L = cap;
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < L; d += (int64_t)gridDim.x * blockDim.x)
        ftab[d] = d > 1 ? (double)d * log((double)d) : 0.0;
}

// ------------------------------------------------------------ exclusive scan
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER;

// Block-wide exclusive scan of one int per thread (all threads must call).
__device__ __forceinline__ int block_exclusive_scan(int x) {
    __shared__ int s_w[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        int t = lane < nw ? s_w[lane] : 0;
        int ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, ti, o);
            if (lane >= o) ti += y;
        }
        s_w[lane] = ti - t;   // exclusive offset of each warp
    }
    __syncthreads();
    int off = s_w[w];
    __syncthreads();
    return off + inc - x;
}

__global__ void k_scan_reduce(const int32_t *__restrict__ in, int32_t n, int32_t *__restrict__ bsum) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        int64_t idx = base + (int64_t)threadIdx.x * SCAN_PER + i;
        if (idx < n) s += in[idx];
    }
    s = warp_sum(s);
    __shared__ int s_w[32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int t = threadIdx.x < (blockDim.x >> 5) ? s_w[threadIdx.x] : 0;
        t = warp_sum(t);
        if (threadIdx.x == 0) bsum[blockIdx.x] = t;
    }
}

// Single block: exclusive scan of the nb block sums in place.
__global__ void k_scan_bsums(int32_t *__restrict__ bsum, int32_t nb) {
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int32_t c0 = 0; c0 < nb; c0 += blockDim.x) {
        int i = c0 + threadIdx.x;
        int x = i < nb ? bsum[i] : 0;
        int ex = block_exclusive_scan(x);
        int carry = s_carry;
        if (i < nb) bsum[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = carry + ex + x;
        __syncthreads();
    }
}

__global__ void k_scan_apply(const int32_t *__restrict__ in, int32_t *__restrict__ out, int32_t n,
                             const int32_t *__restrict__ bsum) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER;
    int v[SCAN_PER];
    int s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    int ex = block_exclusive_scan(s) + bsum[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
        if (base + i == (int64_t)n - 1) out[n] = ex;
    }
}

int launch_scan(const int32_t *in, int32_t *out, int32_t n, int32_t *tmp, cudaStream_t st) {
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int32_t), st) == cudaSuccess ? 0 : -1;
    int32_t nb = (int32_t)((n + SCAN_TILE - 1) / SCAN_TILE);
    k_scan_reduce<<<nb, SCAN_THREADS, 0, st>>>(in, n, tmp);
    k_scan_bsums<<<1, SCAN_THREADS, 0, st>>>(tmp, nb);
    k_scan_apply<<<nb, SCAN_THREADS, 0, st>>>(in, out, n, tmp);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_ftab(double *ftab, const int32_t *maxdeg_dev, int64_t cap, cudaStream_t st) {
    int64_t blocks = (cap + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_ftab<<<(unsigned)blocks, 256, 0, st>>>(ftab, maxdeg_dev, cap);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

static inline unsigned grid_for(int64_t work, int per_block, int64_t cap) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// Validation, degrees, neighbour sums, out-degrees and bins.
int launch_prep_a(const int32_t *rp, const int32_t *ci, int32_t n, int64_t m, const Scratch &s, cudaStream_t st) {
    k_degrees<<<grid_for(n, 256, 1 << 30), 256, 0, st>>>(rp, n, m, s.D, s.counters);
    k_row_stats<<<grid_for(n, 8, 152 * 64), 256, 0, st>>>(rp, ci, n, m, s.D, s.sig1, s.sig2, s.outdeg, s.counters);
    k_bin<<<grid_for(n, 1024, 1 << 30), 1024, 0, st>>>(s.D, s.outdeg, n, s.bins, s.counters);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Oriented CSR, reverse slots, omega, big-item offsets.
int launch_prep_b(const int32_t *rp, const int32_t *ci, int32_t n, int64_t m, const Scratch &s, cudaStream_t st) {
    if (launch_scan(s.outdeg, s.out_ptr, n, s.scan_tmp, st)) return -1;
    k_rev_fill<<<grid_for(n, 8, 152 * 64), 256, 0, st>>>(rp, ci, n, m, s.D, s.sig1, s.out_ptr, s.rev, s.out_col, s.out_D,
                                                         s.out_rslot, s.omega, s.counters);
    // outdeg is free after the scan: reuse it for the big-item counts
    k_big_chunks<<<grid_for(n, 256, 1 << 30), 256, 0, st>>>(s.D, s.bins + (size_t)BIN_BIG * n, s.counters, n, s.outdeg);
    if (launch_scan(s.outdeg, s.big_chunks, n, s.scan_tmp, st)) return -1;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
