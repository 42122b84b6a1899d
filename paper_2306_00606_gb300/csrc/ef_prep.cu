// Preparation passes of libef: CSR validation (with the symmetry sum),
// degrees and work bins, neighbour-degree sums, degree
// orientation for triangle listing, the f(d) = d ln d table, and a
// device-wide exclusive scan.
//
// Algorithm 1's Phase 2 needs |Adj(x)| of every cluster member; the degree
// array D is the only per-node quantity the wedge pass reads besides the CSR.
//
// Row passes use three granularities so that no row's latency chain becomes
// the tail of the pass: a thread per row of degree <= row_thread_max (32 by
// default; loop unrolled by four), a warp per row up to hub_min - 1 (512 by
// default), and a CTA per hub row (listed by the degree kernel, largest
// first).  Both limits are launch parameters (Tune).
#include "ef_internal.cuh"

namespace ef {

// ------------------------------------------------------- block reductions
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *s_buf) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s_buf[w] = v;
    __syncthreads();
    if (w == 0) {
        T t = lane < (int)(blockDim.x >> 5) ? s_buf[lane] : (T)0;
        t = warp_sum(t);
        if (lane == 0) s_buf[0] = t;
    }
    __syncthreads();
    T r = s_buf[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ int64_t block_max_i64(int64_t v, int64_t *s_buf) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, (int64_t)__shfl_xor_sync(FULL, (long long)v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s_buf[w] = v;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < (int)(blockDim.x >> 5) ? s_buf[lane] : INT64_MIN;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = max(t, (int64_t)__shfl_xor_sync(FULL, (long long)t, o));
        if (lane == 0) s_buf[0] = t;
    }
    __syncthreads();
    const int64_t r = s_buf[0];
    __syncthreads();
    return r;
}

// Block-wide exclusive scan of one int per thread (all threads must call).
__device__ __forceinline__ int block_exclusive_scan(int x, int *total = nullptr) {
    __shared__ int s_w[33];
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
        if (lane == 31) s_w[32] = ti;
    }
    __syncthreads();
    int off = s_w[w];
    if (total) *total = s_w[32];
    __syncthreads();
    return off + inc - x;
}

// --------------------------------------------------------- degrees + bins
// A slot in bin b (b < 0: none) of the block's counts s_cnt: the lanes of a
// warp with the same bin take consecutive slots from one atomic.
__device__ __forceinline__ int warp_bin_slot(int *s_cnt, int b) {
    const unsigned want = __ballot_sync(FULL, b >= 0);
    int p = 0;
    if (b >= 0) {
        const unsigned peers = __match_any_sync(want, b);
        const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
        int first = 0;
        if (lane == leader) first = atomicAdd(&s_cnt[b], __popc(peers));
        first = __shfl_sync(peers, first, leader);
        p = first + __popc(peers & ((1u << lane) - 1u));
    }
    return p;
}

// D, max degree, row_ptr checks, and the wedge bins (they depend on D
// only): small sub-warp bins, or "big" plus the mid list or a hub bucket.
// A thread takes DEG_PER nodes, blockDim apart; block-level counting in
// shared memory, one global atomic per bin per block.  (A node per thread in
// blocks of 1024 ran in waves of tiny blocks whose phases -- loads, shared
// counts, global slot atomics, stores -- did not overlap: 0.37 ms for the
// WS batch's 41M nodes.)
constexpr int DEG_THREADS = 256, DEG_PER = 8;

__global__ void __launch_bounds__(DEG_THREADS) k_degrees(const int32_t *__restrict__ rp, int32_t n, int64_t m,
                                                         int hub_min, int32_t *__restrict__ D,
                                                         int32_t *__restrict__ bins, int32_t *__restrict__ cnt) {
    __shared__ int s_cnt[NUM_BINS], s_base[NUM_BINS];
    __shared__ int s_mx[32], s_err[32], s_blo[32], s_bhi[32];
    if (threadIdx.x < NUM_BINS) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t v0 = (int64_t)blockIdx.x * DEG_THREADS * DEG_PER + threadIdx.x;
    int mx = 0, err = 0, blo = 0, bhi = 0;
    int ra[DEG_PER], rb[DEG_PER];
#pragma unroll
    for (int q = 0; q < DEG_PER; ++q) {
        const int64_t v = v0 + q * DEG_THREADS;
        ra[q] = v < n ? rp[v] : 0;
        rb[q] = v < n ? rp[v + 1] : 0;
    }
    int b0[DEG_PER], b1[DEG_PER];
#pragma unroll
    for (int q = 0; q < DEG_PER; ++q) {
        const int64_t v = v0 + q * DEG_THREADS;
        b0[q] = -1;
        b1[q] = -1;
        if (v < n) {
            const int a = ra[q], b = rb[q];
            int d = 0;
            if (a < 0 || b < a || (int64_t)b > m) err |= ERRB_ROWPTR;
            else d = b - a;
            D[v] = d;
            mx = max(mx, d);
            if (d >= 1 && d <= SMALL_MAX) {
                b0[q] = d <= 4 ? BIN_S4 : d <= 8 ? BIN_S8 : d <= 16 ? BIN_S16 : BIN_S32;
            } else if (d > SMALL_MAX) {
                b0[q] = BIN_BIG;
                blo = max(blo, (int)(n - 1 - v));
                bhi = max(bhi, (int)v);
                if (d < hub_min) {
                    b1[q] = BIN_MID;
                } else {
                    const int lg = 31 - __clz(d);   // floor(log2 d)
                    b1[q] = BIN_HUB0 + max(0, min(lg - 9, NUM_HUB_BUCKETS - 1));
                }
            }
        }
    }
    if (v0 == 0 && (rp[0] != 0 || (int64_t)rp[n] != m)) err |= ERRB_ROWPTR;
    // positions in the block's bins: one shared atomic per bin and warp
    // (lattices put a whole block in one or two bins); bin << 16 | position
    // (< DEG_THREADS * DEG_PER), or -1
#pragma unroll
    for (int q = 0; q < DEG_PER; ++q) {
        const int p0 = warp_bin_slot(s_cnt, b0[q]), p1 = warp_bin_slot(s_cnt, b1[q]);
        b0[q] = b0[q] >= 0 ? b0[q] << 16 | p0 : -1;
        b1[q] = b1[q] >= 0 ? b1[q] << 16 | p1 : -1;
    }
    mx = __reduce_max_sync(FULL, mx);
    err = __reduce_or_sync(FULL, err);
    blo = __reduce_max_sync(FULL, blo);
    bhi = __reduce_max_sync(FULL, bhi);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        s_mx[w] = mx;
        s_err[w] = err;
        s_blo[w] = blo;
        s_bhi[w] = bhi;
    }
    __syncthreads();
    if (threadIdx.x < NUM_BINS)
        s_base[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(cnt + threadIdx.x, s_cnt[threadIdx.x]) : 0;
    if (w == 0) {
        // one global atomic per statistic and block (the same few addresses
        // for every block: per-warp atomics there cost 0.07 ms at n = 4M)
        constexpr int nw = DEG_THREADS / 32;
        mx = __reduce_max_sync(FULL, l < nw ? s_mx[l] : 0);
        err = __reduce_or_sync(FULL, l < nw ? s_err[l] : 0);
        blo = __reduce_max_sync(FULL, l < nw ? s_blo[l] : 0);
        bhi = __reduce_max_sync(FULL, l < nw ? s_bhi[l] : 0);
        if (l == 0) {
            if (mx) atomicMax(cnt + CNT_MAXDEG, mx);
            if (err) atomicOr(cnt + CNT_ERR, err);
            if (blo) atomicMax(cnt + CNT_BIGLO, blo);
            if (bhi) atomicMax(cnt + CNT_BIGHI, bhi);
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < DEG_PER; ++q) {
        const int v = (int)(v0 + q * DEG_THREADS);
        if (b0[q] >= 0) bins[(size_t)(b0[q] >> 16) * n + s_base[b0[q] >> 16] + (b0[q] & 0xffff)] = v;
        if (b1[q] >= 0) bins[(size_t)(b1[q] >> 16) * n + s_base[b1[q] >> 16] + (b1[q] & 0xffff)] = v;
    }
}

// Row order of the one-thread row passes (k_row_stats, k_orient), decided on
// the device from the degree pass's counts when the host allows it
// (rows_in_bins_allowed).  When the graph has rows of degree > 32 (degrees
// spread out), the rows of degree 1..32 are taken in work-bin order (the
// lists of degree classes 1-4, 5-8, 9-16 and 17-32 one after the other), so
// that the 32 rows of a warp have similar lengths, and the rows of degree
// 33..hub_min-1 from their list, a warp each.  Otherwise (lattices,
// small-world graphs) they go in node order, where neighbouring rows share
// cache lines.  Measured: BA n = 1M orientation 0.36 -> 0.25 ms in bin
// order; the 4096-graph WS batch 4.7 -> 5.7 ms, so it keeps node order.
struct RowOrder {
    int base[5];   // bin order: first position of each small class, then their total
    bool bins;
    __device__ __forceinline__ void load(const int32_t *cnt, int32_t n, bool allowed) {
        bins = allowed && cnt[BIN_BIG] > 0;
        int acc = 0;
        for (int q = 0; q < 4; ++q) {
            base[q] = acc;
            acc += cnt[BIN_S4 + q];
        }
        base[4] = bins ? acc : n;
    }
    __device__ __forceinline__ int total() const { return base[4]; }
    __device__ __forceinline__ int node(const int32_t *bins_, int32_t n, int i) const {
        if (!bins) return i;
        int q = 0;
        while (base[q + 1] <= i) ++q;
        return bins_[(size_t)(BIN_S4 + q) * n + (i - base[q])];
    }
};

// ------------------------------------------- per-row checks and neighbour sums
// Range, self-loop and strict-order checks; sigma1 = sum of neighbour degrees,
// sigma2 = sum of their squares, and the out-degree in (degree, id) order.
//
// Symmetry check: every entry adds edge_print(v, x) to a per-thread sum,
// reduced per warp into the global symmetry sum (counters[CNT_SYM]), which
// is 0 for a symmetric CSR; the host reads it with the validation word.
struct RowStats {
    int64_t s1 = 0, s2 = 0;
    uint64_t sym = 0;
    int od = 0, err = 0;
    __device__ __forceinline__ void entry(const int32_t *__restrict__ ci, const int32_t *__restrict__ D, int32_t n,
                                          int v, int Dv, int a, int e, NodeMix mv) {
        const int x = ci[e];
        if (x < 0 || x >= n) { err |= ERRB_RANGE; return; }
        if (x == v) err |= ERRB_SELFLOOP;
        if (e > a && ci[e - 1] >= x) err |= ERRB_UNSORTED;
        const int Dx = D[x];
        s1 += Dx;
        s2 += (int64_t)Dx * Dx;
        od += rank_less(Dv, v, Dx, x);
        sym += edge_print(mv, node_mix(x));
    }
    // A whole short row by one thread, four entries at a time: their loads
    // are issued together, so four dependent chains are in flight.
    __device__ __forceinline__ void row(const int32_t *__restrict__ ci, const int32_t *__restrict__ D, int32_t n,
                                        int v, int Dv, int a, int b) {
        const NodeMix mv = node_mix(v);
        int prev = 0;
        for (int e0 = a; e0 < b; e0 += 4) {
            int x[4], Dx[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = e0 + q < b ? ci[e0 + q] : 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) Dx[q] = e0 + q < b && x[q] >= 0 && x[q] < n ? D[x[q]] : 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (e0 + q < b) {
                    const int xq = x[q];
                    const bool later = e0 + q > a;
                    const int before = prev;
                    prev = xq;
                    if (xq < 0 || xq >= n) {
                        err |= ERRB_RANGE;
                        continue;
                    }
                    if (xq == v) err |= ERRB_SELFLOOP;
                    if (later && before >= xq) err |= ERRB_UNSORTED;
                    s1 += Dx[q];
                    s2 += (int64_t)Dx[q] * Dx[q];
                    od += rank_less(Dv, v, Dx[q], xq);
                    sym += edge_print(mv, node_mix(xq));
                }
            }
        }
    }
};

struct RowOut {
    int64_t *sig1, *sig2;
    int32_t *outdeg;
    const int64_t *goff;   // batched input: G + 1 node offsets of the graphs (else nullptr)
    int32_t G;
};

// Batched input: every entry of row v must lie in v's own graph
// [goff[g], goff[g + 1]).  The row pass checks that rows ascend, so the
// first and last entries decide (a < b).
__device__ __forceinline__ int cross_bits(const RowOut &ro, const int32_t *__restrict__ ci, int64_t v, int a, int b) {
    if (!ro.goff || b <= a) return 0;
    int lo = 0, hi = ro.G - 1;   // last g with goff[g] <= v
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ro.goff[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return ci[a] < ro.goff[lo] || ci[b - 1] >= ro.goff[lo + 1] ? ERRB_CROSS : 0;
}

__device__ __forceinline__ void add_sym(int32_t *cnt, uint64_t sym) {
    sym = warp_sum(sym);
    if ((threadIdx.x & 31) == 0 && sym)
        atomicAdd(reinterpret_cast<unsigned long long *>(cnt + CNT_SYM), (unsigned long long)sym);
}

// A row of the row pass walked by a whole warp.
__device__ __forceinline__ void row_stats_warp(const int32_t *__restrict__ ci, const int32_t *__restrict__ D,
                                               int32_t n, int u, int ua, int ub, int lane, const RowOut &ro,
                                               int32_t *__restrict__ cnt, uint64_t &sym) {
    RowStats r;
    const NodeMix mu = node_mix(u);
    for (int e = ua + lane; e < ub; e += 32) r.entry(ci, D, n, u, ub - ua, ua, e, mu);
    const int64_t s1 = warp_sum(r.s1), s2 = warp_sum(r.s2);
    const int od = warp_sum(r.od);
    const int err = __reduce_or_sync(FULL, r.err);
    sym += r.sym;
    if (lane == 0) {
        ro.sig1[u] = s1;
        ro.sig2[u] = s2;
        ro.outdeg[u] = od;
        const int e2 = err | cross_bits(ro, ci, u, ua, ub);
        if (e2) atomicOr(cnt + CNT_ERR, e2);
    }
}

// Rows of degree < hub_min (RowOrder): a thread per row of degree <= tmax,
// the warp for the others; hubs go to k_row_stats_hub.
__global__ void __launch_bounds__(256, 6) k_row_stats(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                      int32_t n, int64_t m, int tmax, int hub_min,
                                                      const int32_t *__restrict__ D, const int32_t *__restrict__ bins,
                                                      bool bins_ok, RowOut ro, int32_t *__restrict__ cnt) {
    __shared__ RowOrder s_ord;
    if (threadIdx.x == 0) s_ord.load(cnt, n, bins_ok);
    __syncthreads();
    const RowOrder &ord = s_ord;
    const int total = ord.total();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    uint64_t sym = 0;
    for (int64_t base = warp * 32; base < total; base += nwarps * 32) {
        const int i = (int)(base + lane);
        const bool in = i < total;
        const int v = in ? ord.node(bins, n, i) : 0;
        const int a = in ? rp[v] : 0, b = in ? rp[v + 1] : 0;
        const bool ok = in && a >= 0 && a <= b && (int64_t)b <= m;
        const int Dv = ok ? b - a : 0;
        if (in && Dv <= tmax) {
            RowStats r;
            if (ok) {
                r.row(ci, D, n, v, Dv, a, b);
                r.err |= cross_bits(ro, ci, v, a, b);
            }
            ro.sig1[v] = r.s1;
            ro.sig2[v] = r.s2;
            ro.outdeg[v] = r.od;
            sym += r.sym;
            if (r.err) atomicOr(cnt + CNT_ERR, r.err);
        }
        unsigned wide = __ballot_sync(FULL, Dv > tmax && Dv < hub_min);
        while (wide) {
            const int j = __ffs(wide) - 1;
            wide &= wide - 1;
            const int u = __shfl_sync(FULL, v, j);
            const int ua = __shfl_sync(FULL, a, j), ub = __shfl_sync(FULL, b, j);
            row_stats_warp(ci, D, n, u, ua, ub, lane, ro, cnt, sym);
        }
    }
    if (ord.bins) {
        const int nmid = cnt[BIN_MID];
        for (int64_t it = warp; it < nmid; it += nwarps) {
            const int u = bins[(size_t)BIN_MID * n + it];
            const int ua = rp[u], ub = rp[u + 1];
            if (ua >= 0 && ua <= ub && (int64_t)ub <= m) row_stats_warp(ci, D, n, u, ua, ub, lane, ro, cnt, sym);
        }
        // rows of degree 0 (or with a malformed range) are in no work list
        for (int64_t v = warp * 32 + lane; v < n; v += nwarps * 32) {
            if (D[v] == 0) {
                ro.sig1[v] = 0;
                ro.sig2[v] = 0;
                ro.outdeg[v] = 0;
            }
        }
    }
    add_sym(cnt, sym);
}

__global__ void __launch_bounds__(ROW_CTA) k_row_stats_hub(const int32_t *__restrict__ rp,
                                                           const int32_t *__restrict__ ci, int32_t n,
                                                           const int32_t *__restrict__ D,
                                                           const int32_t *__restrict__ bins, RowOut ro,
                                                           int32_t *__restrict__ cnt) {
    __shared__ int64_t s_buf[32];
    const int total = hub_total(cnt);
    uint64_t sym = 0;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int u = hub_row(bins, n, cnt, it);
        const int a = rp[u], b = rp[u + 1];
        RowStats r;
        const NodeMix mu = node_mix(u);
        for (int e = a + threadIdx.x; e < b; e += ROW_CTA) r.entry(ci, D, n, u, b - a, a, e, mu);
        const int64_t s1 = block_sum<int64_t>(r.s1, s_buf);
        const int64_t s2 = block_sum<int64_t>(r.s2, s_buf);
        const int64_t od = block_sum<int64_t>(r.od, s_buf);
        const int err = __reduce_or_sync(FULL, r.err);
        sym += r.sym;
        if ((threadIdx.x & 31) == 0 && err) atomicOr(cnt + CNT_ERR, err);
        if (threadIdx.x == 0) {
            ro.sig1[u] = s1;
            ro.sig2[u] = s2;
            ro.outdeg[u] = (int32_t)od;
            if (const int e2 = cross_bits(ro, ci, u, a, b)) atomicOr(cnt + CNT_ERR, e2);
        }
    }
    add_sym(cnt, sym);
}

// ------------------------------------------------------------- orientation
// Appends the out-neighbours x of u (in (degree, id) order) to the oriented
// CSR in ascending id order, with D_x, the probe descriptor of x's own
// out-list and the owner u; and gathers omega_u = sum over N(u) of
// sigma1(x), the last per-node sum the closed form of S needs.  A row walked
// by one thread (at most SMALL_MAX entries, so a table of at most 64 slots)
// also inserts its keys into its hash table, placed with an occupancy mask in
// a register, without atomics; the longer rows' tables are filled afterwards
// by k_hash_rows.  (Atomic inserts inside the warp and block paths made the
// orientation wait one L2 round trip per 32-entry chunk: 0.3 ms more on the
// 4M-node power-law graph.)
static_assert(SMALL_MAX <= 32, "a one-thread row's table fits a 64-bit occupancy mask");
struct OrientStage;
struct Orient {
    const int32_t *ci;
    const int4 *info;   // per node {D, sigma1, probe descriptor of its out-list}
    int32_t *out_col, *out_D, *out_src;
    int2 *out_pd;
    int32_t *out_hash;      // null: no tables
    int32_t *nmin, *nmax;   // optional: smallest / largest neighbour degree (node features)
    int32_t n;
    // u's table from its descriptor (kind 1), when tables are built
    __device__ __forceinline__ bool table(int u, int64_t &base, int &nb) const {
        if (!out_hash) return false;
        const int4 iu = __ldg(info + u);
        base = 4 * (int64_t)iu.z;
        nb = iu.w & DESC_MASK;
        return ((unsigned)iu.w >> DESC_KIND_SHIFT) == 1u;
    }
    __device__ __forceinline__ int4 node(int x) const {
        return x >= 0 && x < n ? __ldg(info + x) : make_int4(0, 0, 0, 0);
    }
    __device__ __forceinline__ bool probe(int u, int Du, int e, int &x, int4 &nf, int64_t &om) const {
        x = ci[e];
        nf = node(x);
        om += nf.y;
        return x >= 0 && x < n && rank_less(Du, u, nf.x, x);
    }
    __device__ __forceinline__ void put(int k, int u, int x, int4 nf) const {
        out_col[k] = x;
        out_D[k] = nf.x;
        out_src[k] = u;
        out_pd[k] = make_int2(nf.z, nf.w);
    }
    // A whole short row by one thread, CHUNK entries at a time (loads issued
    // together); returns omega_v.  With sg, the entries and table keys go to
    // the warp's shared-memory staging area instead (OrientStage).
    template <int CHUNK>
    __device__ __forceinline__ int64_t row(int v, int Dv, int a, int b, int k,
                                           const OrientStage *sg = nullptr) const;
};

// Shared-memory staging of one warp step of one-thread rows: when the rows'
// out-lists form one contiguous range [kbase, kbase + len) of the oriented
// CSR (consecutive rows in layout order, none of them walked elsewhere), the
// rows write their entries and hash-table keys here and the warp then stores
// the range, and its table slots [tbase, tbase + tlen), with coalesced
// stores.  Written directly, a store instruction of 32 rows touched about 12
// sectors for 128 bytes.
struct OrientStage {
    int32_t *col, *D, *src;
    int2 *pd;
    int32_t *tab;
    int kbase;
    int64_t tbase;
    __device__ __forceinline__ void put(int k, int u, int x, int4 nf) const {
        const int i = k - kbase;
        col[i] = x;
        D[i] = nf.x;
        src[i] = u;
        pd[i] = make_int2(nf.z, nf.w);
    }
};

template <int CHUNK>
__device__ __forceinline__ int64_t Orient::row(int v, int Dv, int a, int b, int k, const OrientStage *sg) const {
    {
        int64_t om = 0;
        int mn = 0x7fffffff, mx = 0;
        int64_t hb = 0;
        int nb = 0;
        const bool hashed = table(v, hb, nb);
        const uint64_t full = nb >= 16 ? ~0ull : (1ull << (4 * nb)) - 1ull;
        uint64_t occ = 0;
        for (int e0 = a; e0 < b; e0 += CHUNK) {
            int x[CHUNK];
            int4 nf[CHUNK];
#pragma unroll
            for (int q = 0; q < CHUNK; ++q) x[q] = e0 + q < b ? ci[e0 + q] : -1;
#pragma unroll
            for (int q = 0; q < CHUNK; ++q) nf[q] = node(x[q]);
#pragma unroll
            for (int q = 0; q < CHUNK; ++q) {
                om += nf[q].y;
                if (x[q] >= 0 && x[q] < n) {
                    mn = min(mn, nf[q].x);
                    mx = max(mx, nf[q].x);
                    if (rank_less(Dv, v, nf[q].x, x[q])) {
                        if (sg) sg->put(k++, v, x[q], nf[q]);
                        else put(k++, v, x[q], nf[q]);
                        if (hashed) {
                            // first free slot from the home bucket, cyclically
                            const uint64_t f = ~occ & full;
                            const uint64_t hi = f & (~0ull << (4 * bucket_of(x[q], nb)));
                            const int pos = __ffsll((long long)(hi ? hi : f)) - 1;
                            if (sg) sg->tab[hb + pos - sg->tbase] = x[q];
                            else out_hash[hb + pos] = x[q];
                            occ |= 1ull << pos;
                        }
                    }
                }
            }
        }
        if (nmin) {
            nmin[v] = mx ? mn : 0;
            nmax[v] = mx;
        }
        return om;
    }
}

// info[v] = {D_v, sigma1(v), probe descriptor of v's out-list}: what the
// orientation needs of a neighbour, in one 16-byte gather (sigma1 <= m < 2^31).
__global__ void k_node_info(const int32_t *__restrict__ D, const int64_t *__restrict__ sig1,
                            const int32_t *__restrict__ out_ptr, const int32_t *__restrict__ outdeg, int32_t n,
                            int64_t hash_cap, int4 *__restrict__ info) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int ls = out_ptr[v];
        const int2 pd = probe_desc(ls, ls + outdeg[v], hash_cap);
        info[v] = make_int4(D[v], (int)sig1[v], pd.x, pd.y);
    }
}

// Layout of the oriented CSR: the out-lists are stored work bin by work bin
// (degree classes 1-4, 5-8, 9-16, 17-32, the warp class, the hub buckets),
// not in node order, so that the lists of nodes of similar degree -- and
// similar odds of being probed by the triangle pass -- share cache lines.
// Nodes of degree 0 have no list.
constexpr int LAYOUT_BINS = 5 + NUM_HUB_BUCKETS;
__constant__ int c_layout_bins[LAYOUT_BINS] = {BIN_S4,       BIN_S8,       BIN_S16,      BIN_S32,
                                               BIN_MID,      BIN_HUB0,     BIN_HUB0 + 1, BIN_HUB0 + 2,
                                               BIN_HUB0 + 3, BIN_HUB0 + 4, BIN_HUB0 + 5, BIN_HUB0 + 6};
static_assert(BIN_HUB0 + 6 == BIN_HUB_LAST, "layout bins cover the hub buckets");

// base[q] = first layout position of bin q; base[LAYOUT_BINS] = all listed nodes.
__device__ __forceinline__ void layout_bases(const int32_t *cnt, int *base) {
    int acc = 0;
    for (int q = 0; q < LAYOUT_BINS; ++q) {
        base[q] = acc;
        acc += cnt[c_layout_bins[q]];
    }
    base[LAYOUT_BINS] = acc;
}

// The node at layout position i < base[LAYOUT_BINS].
__device__ __forceinline__ int layout_node(const int32_t *bins, int32_t n, const int *base, int i) {
    int q = 0;
    while (base[q + 1] <= i) ++q;
    return bins[(size_t)c_layout_bins[q] * n + (i - base[q])];
}

__global__ void k_layout_gather(const int32_t *__restrict__ bins, const int32_t *__restrict__ cnt, int32_t n,
                                const int32_t *__restrict__ outdeg, int32_t *__restrict__ lay_node,
                                int32_t *__restrict__ lay_deg) {
    if (gate_closed(cnt)) return;
    __shared__ int s_base[LAYOUT_BINS + 1];
    if (threadIdx.x == 0) layout_bases(cnt, s_base);
    __syncthreads();
    const int total = s_base[LAYOUT_BINS];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i >= total) {
            lay_deg[i] = 0;
            continue;
        }
        const int v = layout_node(bins, n, s_base, i);
        lay_node[i] = v;
        lay_deg[i] = outdeg[v];
    }
}

__global__ void k_layout_scatter(const int32_t *__restrict__ cnt, int32_t n, const int32_t *__restrict__ lay_node,
                                 const int32_t *__restrict__ lay_ptr, int32_t *__restrict__ out_ptr) {
    if (gate_closed(cnt)) return;
    __shared__ int s_base[LAYOUT_BINS + 1];
    if (threadIdx.x == 0) layout_bases(cnt, s_base);
    __syncthreads();
    const int total = s_base[LAYOUT_BINS];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
        out_ptr[lay_node[i]] = lay_ptr[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) out_ptr[n] = lay_ptr[total];
}

// A row walked by a whole warp (degree above tmax, below hub_min).
__device__ __forceinline__ void orient_row_warp(const Orient &o, int u, int ua, int ub, int k0, int lane,
                                                int64_t *__restrict__ omega) {
    int64_t om = 0;
    int mn = 0x7fffffff, mx = 0;
    for (int e0 = ua; e0 < ub; e0 += 32) {
        const int e = e0 + lane;
        int x = 0;
        int4 nf = make_int4(0, 0, 0, 0);
        const bool isout = e < ub && o.probe(u, ub - ua, e, x, nf, om);
        if (e < ub && x >= 0 && x < o.n) {
            mn = min(mn, nf.x);
            mx = max(mx, nf.x);
        }
        const unsigned bal = __ballot_sync(FULL, isout);
        if (isout) o.put(k0 + __popc(bal & ((1u << lane) - 1u)), u, x, nf);
        k0 += __popc(bal);
    }
    om = warp_sum(om);
    mn = __reduce_min_sync(FULL, mn);
    mx = __reduce_max_sync(FULL, mx);
    if (lane == 0) {
        omega[u] = om;
        if (o.nmin) {
            o.nmin[u] = mx ? mn : 0;
            o.nmax[u] = mx;
        }
    }
}

// Rows of degree < hub_min (RowOrder): a thread per row of degree <= tmax,
// the warp for the others; hubs go to k_orient_hub.  A one-thread row gathers
// the records of CHUNK entries at once: 8 (3 blocks per SM) when no row
// exceeds degree 32, 4 (5 blocks per SM) otherwise, where short rows would
// waste most of a wide chunk.  Both forms are launched; the one that does not
// match the degree pass's counts returns at once.  (WS batch orientation
// 4.7 -> 4.3 ms with 8; the power-law graph 0.90 -> 1.02 ms with 8.)
// Entries of one warp step that the staging area of k_orient<CHUNK> holds
// (20 bytes each, plus two table slots).  Only the eight-record form (graphs
// without rows above degree 32) stages: measured on the 4096-graph WS batch,
// orientation 4.32 -> 2.96 ms; the four-record form (a staging area of 128
// entries, 5 blocks per SM) was slower on the power-law graph (0.89 -> 0.96
// ms), BA 16M (2.42 -> 2.55 ms) and BA 1M, where its rows are longer or come
// from the degree bins and the warp's rows rarely fit, so it writes directly.
template <int CHUNK>
struct OrientCap {
    static constexpr int value = CHUNK == 8 ? 192 : 0;
};

template <int CHUNK>
__global__ void __launch_bounds__(256, CHUNK == 8 ? 3 : 5) k_orient(
    const int32_t *__restrict__ rp, int32_t n, int64_t m, int tmax, int hub_min, Orient o,
    const int32_t *__restrict__ D, const int32_t *__restrict__ bins, bool bins_ok, const int32_t *__restrict__ cnt,
    const int32_t *__restrict__ out_ptr, const int32_t *__restrict__ outdeg, int64_t *__restrict__ omega) {
    if (gate_closed(cnt)) return;
    if ((cnt[BIN_BIG] == 0) != (CHUNK == 8)) return;
    constexpr int CAP = OrientCap<CHUNK>::value;
    constexpr int SCAP = CAP > 0 ? CAP : 1, TCAP = CAP > 0 ? 2 * CAP + 8 : 1;
    __shared__ RowOrder s_ord;
    __shared__ int32_t s_col[8][SCAP], s_D[8][SCAP], s_src[8][SCAP], s_tab[8][TCAP];
    __shared__ int2 s_pd[8][SCAP];
    if (threadIdx.x == 0) s_ord.load(cnt, n, bins_ok);
    __syncthreads();
    const RowOrder &ord = s_ord;
    const int total = ord.total();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + w;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = warp * 32; base < total; base += nwarps * 32) {
        const int i = (int)(base + lane);
        const bool in = i < total;
        const int v = in ? ord.node(bins, n, i) : 0;
        const int a = in ? rp[v] : 0, b = in ? rp[v + 1] : 0;
        const bool ok = in && a >= 0 && a <= b && (int64_t)b <= m;
        const int Dv = ok ? b - a : 0;
        const bool mine = ok && Dv <= tmax;
        const int k0 = mine ? out_ptr[v] : 0;
        // stage when this step's one-thread rows own one contiguous range that
        // fits: span of their out-lists == sum of their lengths (no other row's
        // list inside), both within CAP
        int kmin = 0, kend = 0, sum = 0;
        if constexpr (CAP > 0) {
            const int od = mine ? outdeg[v] : 0;
            kmin = __reduce_min_sync(FULL, od > 0 ? k0 : 0x7fffffff);
            kend = __reduce_max_sync(FULL, od > 0 ? k0 + od : 0);
            sum = __reduce_add_sync(FULL, od);
        }
        const bool stage = CAP > 0 && sum > 0 && sum <= CAP && kend - kmin == sum;
        if (stage) {
            const int64_t tb0 = ((int64_t)2 * kmin + 3) & ~(int64_t)3;
            const int64_t tb1 = ((int64_t)2 * kend + 3) & ~(int64_t)3;
            const int tlen = o.out_hash ? (int)(tb1 - tb0) : 0;
            for (int t = lane; t < tlen; t += 32) s_tab[w][t] = -1;
            __syncwarp();
            const OrientStage sg{s_col[w], s_D[w], s_src[w], s_pd[w], s_tab[w], kmin, tb0};
            if (mine) omega[v] = o.template row<CHUNK>(v, Dv, a, b, k0, &sg);
            __syncwarp();
            for (int t = lane; t < sum; t += 32) {
                o.out_col[kmin + t] = s_col[w][t];
                o.out_D[kmin + t] = s_D[w][t];
                o.out_src[kmin + t] = s_src[w][t];
                o.out_pd[kmin + t] = s_pd[w][t];
            }
            for (int t = lane; t < tlen; t += 32) o.out_hash[tb0 + t] = s_tab[w][t];
            __syncwarp();
        } else if (mine) {
            omega[v] = o.template row<CHUNK>(v, Dv, a, b, k0);
        }
        unsigned wide = __ballot_sync(FULL, ok && Dv > tmax && Dv < hub_min);
        while (wide) {
            const int j = __ffs(wide) - 1;
            wide &= wide - 1;
            const int u = __shfl_sync(FULL, v, j);
            const int ua = __shfl_sync(FULL, a, j), ub = __shfl_sync(FULL, b, j);
            orient_row_warp(o, u, ua, ub, out_ptr[u], lane, omega);
        }
    }
    if (!ord.bins) return;
    const int nmid = cnt[BIN_MID];
    for (int64_t it = warp; it < nmid; it += nwarps) {
        const int u = bins[(size_t)BIN_MID * n + it];
        const int ua = rp[u], ub = rp[u + 1];
        if (ua >= 0 && ua <= ub && (int64_t)ub <= m) orient_row_warp(o, u, ua, ub, out_ptr[u], lane, omega);
    }
    // rows of degree 0 are in no work list
    for (int64_t v = warp * 32 + lane; v < n; v += nwarps * 32) {
        if (D[v] == 0) {
            omega[v] = 0;
            if (o.nmin) {
                o.nmin[v] = 0;
                o.nmax[v] = 0;
            }
        }
    }
}

__global__ void __launch_bounds__(ROW_CTA) k_orient_hub(const int32_t *__restrict__ rp, int32_t n, Orient o,
                                                        const int32_t *__restrict__ bins,
                                                        const int32_t *__restrict__ out_ptr,
                                                        const int32_t *__restrict__ cnt,
                                                        int64_t *__restrict__ omega) {
    if (gate_closed(cnt)) return;
    __shared__ int64_t s_buf[32];
    __shared__ int s_k;
    const int total = hub_total(cnt);
    const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int u = hub_row(bins, n, cnt, it);
        const int a = rp[u], b = rp[u + 1];
        // the out-list's entries take their positions from a shared counter,
        // one atomic per warp and pass (no block barrier per pass; the
        // list's order varies, which nothing downstream depends on)
        if (threadIdx.x == 0) s_k = out_ptr[u];
        __syncthreads();
        int64_t om = 0;
        int64_t mn = 0x7fffffff, mx = 0;
        for (int e0 = a; e0 < b; e0 += ROW_CTA) {
            const int e = e0 + threadIdx.x;
            int x = 0;
            int4 nf = make_int4(0, 0, 0, 0);
            const bool isout = e < b && o.probe(u, b - a, e, x, nf, om);
            if (e < b && x >= 0 && x < n) {
                mn = min(mn, (int64_t)nf.x);
                mx = max(mx, (int64_t)nf.x);
            }
            const unsigned bal = __ballot_sync(FULL, isout);
            int wk = 0;
            if ((threadIdx.x & 31) == 0 && bal) wk = atomicAdd(&s_k, __popc(bal));
            wk = __shfl_sync(FULL, wk, 0);
            if (isout) o.put(wk + __popc(bal & lt), u, x, nf);
        }
        om = block_sum<int64_t>(om, s_buf);
        if (o.nmin) {
            // min and max through the sum reduction: -max(-x), max(x)
            mx = block_max_i64(mx, s_buf);
            mn = -block_max_i64(-mn, s_buf);
        }
        if (threadIdx.x == 0) {
            omega[u] = om;
            if (o.nmin) {
                o.nmin[u] = mx ? (int32_t)mn : 0;
                o.nmax[u] = (int32_t)mx;
            }
        }
    }
}

// Hash tables of the rows longer than tmax (walked by a warp or a block in
// the orientation): a warp per such row, its lanes inserting the row's
// out-list entries by atomics.  The rows come from the list of nodes of
// degree > SMALL_MAX when tmax = SMALL_MAX (the default), else from a scan of
// all nodes.
__global__ void k_hash_rows(const int32_t *__restrict__ rp, int32_t n, int64_t m, int tmax,
                            const int32_t *__restrict__ big_list, const int32_t *__restrict__ cnt,
                            const int4 *__restrict__ info, const int32_t *__restrict__ out_ptr,
                            const int32_t *__restrict__ outdeg, const int32_t *__restrict__ out_col,
                            int32_t *__restrict__ out_hash) {
    if (gate_closed(cnt)) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t count = tmax >= SMALL_MAX ? cnt[BIN_BIG] : n;
    for (int64_t i = warp; i < count; i += nwarps) {
        const int u = tmax >= SMALL_MAX ? big_list[i] : (int)i;
        const int a = rp[u], b = rp[u + 1];
        const int4 iu = __ldg(info + u);
        if (!(a >= 0 && a <= b && (int64_t)b <= m && b - a > tmax &&
              ((unsigned)iu.w >> DESC_KIND_SHIFT) == 1u))
            continue;
        const int64_t hb = 4 * (int64_t)iu.z;
        const int nb = iu.w & DESC_MASK;
        const int ls = out_ptr[u], p = outdeg[u];
        for (int e = lane; e < p; e += 32) table_insert_shared(out_hash, hb, nb, out_col[ls + e]);
    }
}

// The same in the degree-bin layout with tmax = SMALL_MAX: the out-lists of
// the rows of degree > SMALL_MAX are the tail of the oriented CSR (the mid
// and hub bins come last), so a thread per entry of that tail inserts it into
// its owner's table.  Independent entries keep many inserts in flight, where
// a warp per row waited on four dependent loads per row.
__global__ void k_hash_tail(const int32_t *__restrict__ cnt, const int32_t *__restrict__ lay_ptr,
                            const int32_t *__restrict__ out_ptr, int32_t n, const int4 *__restrict__ info,
                            const int32_t *__restrict__ out_col, const int32_t *__restrict__ out_src,
                            int32_t *__restrict__ out_hash) {
    if (gate_closed(cnt)) return;
    __shared__ int s_base[LAYOUT_BINS + 1];
    if (threadIdx.x == 0) layout_bases(cnt, s_base);
    __syncthreads();
    const int64_t first = lay_ptr[s_base[4]];   // layout bin 4 = BIN_MID, the first list of degree > SMALL_MAX
    const int64_t total = out_ptr[n];
    for (int64_t k = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int a = out_src[k];
        const int4 ia = __ldg(info + a);
        if (((unsigned)ia.w >> DESC_KIND_SHIFT) == 1u)
            table_insert_shared(out_hash, 4 * (int64_t)ia.z, ia.w & DESC_MASK, out_col[k]);
    }
}

// Work items of the big middle nodes for the direct kernel: ceil(D / BIG_ROWS)
// each; entries past the bin count are 0 so a scan over n gives the offsets.
__global__ void k_big_chunks(const int32_t *__restrict__ D, const int32_t *__restrict__ big_list,
                             const int32_t *__restrict__ cnt, int32_t n, int32_t *__restrict__ chunks) {
    if (gate_closed(cnt)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int nb = cnt[BIN_BIG];
    chunks[i] = i < nb ? (D[big_list[i]] + BIG_ROWS - 1) / BIG_ROWS : 0;
}

// -------------------------------------------------------------- f(d) table
// ftab[d] = d ln d (computed in FP64, stored as the FP32 pair hi + lo of
// F2Sum: hi = f rounded to FP32, lo = the rest rounded to FP32, together
// within 2^-48 of f); tq[s] = 4 (f(s-6) - f(s-4)) in units of 2^-F, the
// correction one triangle of degree sum s brings to each of its nodes.  F is
// the largest value <= TRI_FRAC_MAX with C(maxdeg, 2) * max|g| * 2^F < 2^62
// (|g| <= 8 (ln(3 maxdeg) + 1) + 8); every thread derives the same F and
// thread 0 publishes it for the finalize pass.
__global__ void k_ftab(float2 *__restrict__ ftab, int64_t *__restrict__ tq, int32_t *__restrict__ cnt, int64_t cap) {
    if (gate_closed(cnt)) return;
    const int64_t maxdeg = cnt[CNT_MAXDEG];
    int64_t L = 3 * maxdeg + 1;
    if (L > cap) L = cap;
    // blocks past the table (the grid is sized for the capacity, which may
    // be far above 3 maxdeg + 1 when it was not read back) leave at once
    if ((int64_t)blockIdx.x * blockDim.x >= L && blockIdx.x != 0) return;
    __shared__ int s_F;
    if (threadIdx.x == 0) {
        const double tmax = 0.5 * (double)maxdeg * (double)(maxdeg > 0 ? maxdeg - 1 : 0) + 1.0;
        const double gmax = 8.0 * (log(3.0 * (double)maxdeg + 8.0) + 1.0) + 8.0;
        const int F0 = (int)floor(62.0 - log2(tmax * gmax));
        s_F = F0 > TRI_FRAC_MAX ? TRI_FRAC_MAX : (F0 < 0 ? 0 : F0);
        if (blockIdx.x == 0) cnt[CNT_TRIFRAC] = s_F;
    }
    __syncthreads();
    const int F = s_F;
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < L; d += (int64_t)gridDim.x * blockDim.x) {
        const double f = d > 1 ? (double)d * log((double)d) : 0.0;
        const float hi = (float)f;
        ftab[d] = make_float2(hi, (float)(f - (double)hi));
        double g = 0.0;
        if (d >= 6) {
            const double a = (double)(d - 6), b = (double)(d - 4);
            g = 4.0 * ((a > 1.0 ? a * log(a) : 0.0) - b * log(b));
        }
        tq[d] = llrint(ldexp(g, F));
    }
}

// ------------------------------------------------------------ exclusive scan
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER;

__global__ void k_scan_reduce(const int32_t *__restrict__ in, int32_t n, int32_t *__restrict__ bsum) {
    __shared__ int s_buf[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        int64_t idx = base + (int64_t)threadIdx.x * SCAN_PER + i;
        if (idx < n) s += in[idx];
    }
    s = block_sum<int>(s, s_buf);
    if (threadIdx.x == 0) bsum[blockIdx.x] = s;
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

// in and out may be the same array (each thread reads its own elements
// before it writes them), so they are not __restrict__.
__global__ void k_scan_apply(const int32_t *in, int32_t *out, int32_t n, const int32_t *__restrict__ bsum) {
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

__global__ void k_gate(int32_t *__restrict__ cnt, int32_t *__restrict__ sticky) {
    unsigned long long sym;
    memcpy(&sym, cnt + CNT_SYM, sizeof sym);
    const int bits = cnt[CNT_ERR] | (sym ? ERRB_ASYM : 0) | (cnt[CNT_MAXDEG] > EF_MAX_DEGREE ? ERRB_DEGREE : 0);
    cnt[CNT_GATE] = bits;
    if (bits && sticky) atomicOr(sticky, bits);
}

int launch_gate(int32_t *cnt, int32_t *sticky, cudaStream_t st) {
    k_gate<<<1, 1, 0, st>>>(cnt, sticky);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_ftab(float2 *ftab, int64_t *tq, int32_t *cnt, int64_t cap, cudaStream_t st) {
    int64_t blocks = (cap + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    k_ftab<<<(unsigned)blocks, 256, 0, st>>>(ftab, tq, cnt, cap);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

static inline unsigned grid_for(int64_t work, int per_block, int64_t cap) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// Degrees + wedge bins, per-row checks and neighbour sums.
int launch_prep_a(const int32_t *rp, const int32_t *ci, int32_t n, int64_t m, const Scratch &s, const Tune &t,
                  cudaStream_t st, const int64_t *goff, int32_t G) {
    k_degrees<<<grid_for(n, DEG_THREADS * DEG_PER, 1 << 30), DEG_THREADS, 0, st>>>(rp, n, m, t.hub_min, s.D, s.bins,
                                                                                 s.counters);
    const RowOut ro{s.sig1, s.sig2, s.outdeg, goff, G};
    k_row_stats<<<t.grid((int64_t)n, 256), 256, 0, st>>>(rp, ci, n, m, t.row_thread_max, t.hub_min, s.D, s.bins,
                                                         rows_in_bins_allowed(m), ro, s.counters);
    k_row_stats_hub<<<t.num_sms * 4, ROW_CTA, 0, st>>>(rp, ci, n, s.D, s.bins, ro, s.counters);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Oriented CSR and omega.
int launch_orient(const int32_t *rp, const int32_t *ci, int32_t n, int64_t m, const Scratch &s, const Tune &t,
                  cudaStream_t st, int32_t *nmin, int32_t *nmax, bool bins, bool tables) {
    if (tables && cudaMemsetAsync(s.out_hash, 0xff, (size_t)hash_slots(m) * sizeof(int32_t), st) != cudaSuccess)
        return -1;
    if (bins) {
        // out-list offsets in layout order (degree-0 nodes keep offset 0 and an empty list)
        if (cudaMemsetAsync(s.out_ptr, 0, (size_t)(n + 1) * sizeof(int32_t), st) != cudaSuccess) return -1;
        k_layout_gather<<<t.grid((int64_t)n, 256), 256, 0, st>>>(s.bins, s.counters, n, s.outdeg, s.lay_node,
                                                                 s.lay_ptr);
        if (launch_scan(s.lay_ptr, s.lay_ptr, n, s.scan_tmp, st)) return -1;
        k_layout_scatter<<<t.grid((int64_t)n, 256), 256, 0, st>>>(s.counters, n, s.lay_node, s.lay_ptr, s.out_ptr);
    } else if (launch_scan(s.outdeg, s.out_ptr, n, s.scan_tmp, st)) {
        return -1;
    }
    k_node_info<<<t.grid((int64_t)n, 256), 256, 0, st>>>(s.D, s.sig1, s.out_ptr, s.outdeg, n, hash_slots(m),
                                                         s.info);
    const Orient o{ci, s.info, s.out_col, s.out_D, s.out_src, s.out_pd, tables ? s.out_hash : nullptr, nmin, nmax, n};
    k_orient<4><<<t.grid((int64_t)n, 256), 256, 0, st>>>(rp, n, m, t.row_thread_max, t.hub_min, o, s.D, s.bins,
                                                         rows_in_bins_allowed(m), s.counters, s.out_ptr, s.outdeg,
                                                         s.omega);
    k_orient<8><<<t.grid((int64_t)n, 256), 256, 0, st>>>(rp, n, m, t.row_thread_max, t.hub_min, o, s.D, s.bins,
                                                         rows_in_bins_allowed(m), s.counters, s.out_ptr, s.outdeg,
                                                         s.omega);
    k_orient_hub<<<t.num_sms * 4, ROW_CTA, 0, st>>>(rp, n, o, s.bins, s.out_ptr, s.counters, s.omega);
    if (tables && bins && t.row_thread_max >= SMALL_MAX)
        k_hash_tail<<<(unsigned)(t.num_sms * 16), 256, 0, st>>>(s.counters, s.lay_ptr, s.out_ptr, n, s.info,
                                                               s.out_col, s.out_src, s.out_hash);
    else if (tables)
        k_hash_rows<<<(unsigned)(t.num_sms * 8), 256, 0, st>>>(rp, n, m, t.row_thread_max, s.bins + (size_t)BIN_BIG * n,
                                                               s.counters, s.info, s.out_ptr, s.outdeg, s.out_col,
                                                               s.out_hash);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Item offsets of the direct big-node wedge kernel (counts, then an in-place
// scan with its own block-sum buffer: it may run beside the orientation).
int launch_big_items(const Scratch &s, int32_t n, cudaStream_t st) {
    k_big_chunks<<<grid_for(n, 256, 1 << 30), 256, 0, st>>>(s.D, s.bins + (size_t)BIN_BIG * n, s.counters, n,
                                                             s.big_chunks);
    if (launch_scan(s.big_chunks, s.big_chunks, n, s.scan_tmp2, st)) return -1;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
