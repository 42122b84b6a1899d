// Triangle pass of libef (Algorithm 1, Phase 2: the "i in Adj(j)" test).
//
// The wedge pass credits every cluster with its open degree; clusters whose
// ends are adjacent (triangles) need d - 2 instead.  Edges are oriented from
// lower to higher (degree, id); each triangle is found exactly once, at its
// lowest-ranked node a, as an adjacent pair {b, c} of a's out-neighbours
// N+(a) (b before c in N+(a)'s id order).  Its three nodes each hold 4
// credits of degree sum-6 that the wedge pass counted at sum-4
// (sum = D_a + D_b + D_c), so each receives g = 4 (f(sum-6) - f(sum-4)) and
// one triangle count.
//
// Pair tests: b and c are adjacent iff the higher-ranked of the two is in the
// lower-ranked one's out-list.  That is sum_a C(|N+(a)|, 2) independent tests
// -- 1.1e8 on the 4M-node power-law workload, against 1.15e9 dependent steps
// for merging the two out-lists of every edge.  A warp takes 64 consecutive
// oriented edges, cuts each edge's candidates c into units of TRI_UNIT and
// spreads the units evenly over its lanes.
//
// The pass is bound by L2 latency, so every membership test is one round of
// two independent 16-byte loads, the same instructions for every lane: an
// out-list of at most SHORT_MAX entries is read whole (it spans at most two
// aligned quads); a longer one has a bucketed hash table (4 slots per
// 16-byte bucket, load factor <= 0.5 + small rounding, built by the orientation)
// and the key's bucket and the next one are loaded together, which settles
// the test but for rare long probe runs.  The oriented CSR carries, for each
// out-neighbour, the probe descriptor of its own list (which quads to load
// and how to read them, fixed once per node by the orientation), so no test
// waits for an out_ptr load or recomputes a table's geometry.
//
// Measured and left out (4M-node power-law graph): L2 eviction hints
// (evict_last on probes, evict_first on the candidate stream) changed
// nothing; staging each tile's candidates in shared memory was slower
// (2.00 against 1.84 ms, and again 1.74 against 1.65 ms with a warp step's
// 128 entries staged by coalesced loads); loading each test's correction
// tq[sum] with its probes, to save the second round trip of a hit, was
// slower too (1.85 against 1.65 ms; the per-unit binary search replaced by
// a shared-memory unit map changed nothing).  Under ncu (half-size graph)
// the kernel issues in 46% of cycles, waits on long-scoreboard loads (7.2
// cycles per issue) with 39% of the warp slots filled (64 registers), and
// uses 31% of L2 and 8% of DRAM throughput: bound by the latency of its
// probes at the concurrency its registers allow.  The pass reads about 1.5 GB from DRAM per launch,
// mostly misses of the long tail of membership probes (10% of the tests spread
// over about 100 MB of tables and lists).
//
// The pass is integer-only: g comes from a table in fixed point (units of
// 2^-F, F chosen per call from the maximum degree), so the sums are exact and
// independent of the order of the atomics, and no FP64 instruction (one lane
// per clock per SM sub-partition on this GPU) sits in a divergent branch.
// Corrections and counts go to per-node accumulators (qacc, tcnt) by L2
// reductions: c's at once, b's once per unit, a's merged per lane over
// consecutive units of the same owner.
//
// A shard of the pass lists the triangles whose lowest-ranked node lies in
// its node range (a node id range: the oriented layout's list order comes
// from atomics and differs between calls, node ids and ranks do not).
#include "ef_internal.cuh"

namespace ef {

constexpr int TRI_WARPS = 8;
// Kernel variants: candidate pairs per lane step (TRI_UNIT), resident blocks
// per SM the registers are sized for, and oriented edges per warp step (EW).
// Measured on the 4M-node power-law graph with EW = 32: (2, 4) 1.80 ms,
// (2, 3) 1.98, (2, 5) 2.06, (4, 3) 2.28, (4, 4) 2.51 (register spills).
// EW = 64 fills the last round of a step better where out-lists are short:
// WS batch 6.13 -> 5.65 ms, BA 1M 0.174 -> 0.154, power-law 1.665 -> 1.653.
// Variant 0 = (2, 4, 64), 1 = (4, 3, 32).

__device__ __forceinline__ unsigned match4(int4 v, int key) {
    return (unsigned)(v.x == key) | (unsigned)(v.y == key) << 1 | (unsigned)(v.z == key) << 2 |
           (unsigned)(v.w == key) << 3;
}

__device__ __forceinline__ bool has_empty(int4 v) { return (v.x | v.y | v.z | v.w) < 0; }

// One membership test "key in the out-list of probe descriptor pd", split so
// that a lane issues the loads of all its tests before it waits for any: the
// quads p0 and p0 + d1, and which of their entries count (info bits 0-3 and
// 4-7) and the kind of list (bits 8-9, the descriptor's kind).
struct Probe {
    const int4 *p0;
    int d1;
    unsigned info;
};

__device__ __forceinline__ Probe probe_of(const int32_t *out_col, const int32_t *out_hash, int2 pd, int key) {
    Probe r;
    const unsigned kind = (unsigned)pd.y >> DESC_KIND_SHIFT;
    if (kind == 1) {
        const int nb = pd.y & DESC_MASK;
        const int b0 = bucket_of(key, nb);
        r.p0 = reinterpret_cast<const int4 *>(out_hash) + ((int64_t)pd.x + b0);
        r.d1 = b0 + 1 == nb ? -b0 : 1;
        r.info = 0xffu | 1u << 8;
    } else if (kind == 0) {
        r.p0 = reinterpret_cast<const int4 *>(out_col) + pd.x;
        r.d1 = 1;
        r.info = (unsigned)pd.y & 0xffu;
    } else {
        r.p0 = reinterpret_cast<const int4 *>(out_col) + (pd.x >> 2);
        r.d1 = 1;
        r.info = 2u << 8;
    }
    return r;
}

// Resolve a probe from its two loaded quads.  The rare ends -- a hashed probe
// whose two buckets were full without the key (continue the run), a long
// list without a table (malformed input only: binary search) -- reload what
// they need.
__device__ __forceinline__ bool probe_done(const Probe &r, int4 x, int4 y, const int32_t *out_col,
                                           const int32_t *out_hash, int2 pd, int key) {
    if ((match4(x, key) & r.info) | (match4(y, key) & (r.info >> 4) & 0xfu)) return true;
    const unsigned kind = (r.info >> 8) & 3u;
    if (kind == 0 || (kind == 1 && (has_empty(x) || has_empty(y)))) return false;
    if (kind == 1) {
        const int nb = pd.y & DESC_MASK;
        const int4 *t = reinterpret_cast<const int4 *>(out_hash) + pd.x;
        int b = (int)(r.p0 + r.d1 - t);
        b = b + 1 == nb ? 0 : b + 1;
        for (int tries = 2; tries < nb; ++tries) {
            const int4 q = __ldg(t + b);
            if (match4(q, key)) return true;
            if (has_empty(q)) return false;
            b = b + 1 == nb ? 0 : b + 1;
        }
        return false;
    }
    const int ls = pd.x, le = pd.y & DESC_MASK;
    const int pos = ls + lower_bound_i32(out_col + ls, le - ls, key);
    return pos < le && out_col[pos] == key;
}

__device__ __forceinline__ void credit_tri(int64_t *qacc, int64_t *tcnt, int v, int64_t q, int cnt) {
    atomicAdd((unsigned long long *)(qacc + v), (unsigned long long)q);
    atomicAdd((unsigned long long *)(tcnt + v), (unsigned long long)cnt);
}

template <int TRI_UNIT, int TRI_BLOCKS, int EW>
__global__ void __launch_bounds__(TRI_WARPS * 32, TRI_BLOCKS) k_tri_pairs(
    const int32_t *__restrict__ out_ptr, const int32_t *__restrict__ out_col, const int32_t *__restrict__ out_D,
    const int2 *__restrict__ out_pd, const int32_t *__restrict__ out_src, const int32_t *__restrict__ out_hash,
    const int32_t *__restrict__ outdeg, const int32_t *__restrict__ D, int32_t n,
    const int32_t *__restrict__ owner_range, const int64_t *__restrict__ tq,
    int64_t *__restrict__ qacc, int64_t *__restrict__ tcnt, const int32_t *__restrict__ cnt) {
    static_assert(EW == 32 || EW == 64, "a warp step takes 32 or 64 edges");
    __shared__ int s_ex[TRI_WARPS][EW];   // exclusive prefix of unit counts
    __shared__ int s_kend[TRI_WARPS][EW], s_b[TRI_WARPS][EW], s_Db[TRI_WARPS][EW], s_Dab[TRI_WARPS][EW];
    __shared__ int s_a[TRI_WARPS][EW];
    __shared__ int2 s_bpd[TRI_WARPS][EW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t total = gate_closed(cnt) ? 0 : out_ptr[n];   // no pairs when the device check failed
    const int64_t stride = (int64_t)gridDim.x * TRI_WARPS * EW;
    // owners a in [a_lo, a_hi) open their pairs (all nodes, or one shard's range)
    const int a_lo = owner_range ? owner_range[0] : 0, a_hi = owner_range ? owner_range[1] : n;
    for (int64_t K0 = ((int64_t)blockIdx.x * TRI_WARPS + w) * EW; K0 < total; K0 += stride) {
        int U = 0;
#pragma unroll
        for (int h = 0; h < EW / 32; ++h) {
            const int e = h * 32 + lane;
            const int64_t k = K0 + e;
            int nu = 0;
            if (k < total) {
                const int a = out_src[k];
                const int kend = out_ptr[a] + outdeg[a];
                const int np = a >= a_lo && a < a_hi ? kend - (int)k - 1 : 0;
                if (np > 0) {
                    const int b = out_col[k];
                    const int Db = out_D[k];
                    s_kend[w][e] = kend;
                    s_b[w][e] = b;
                    s_Db[w][e] = Db;
                    s_bpd[w][e] = out_pd[k];
                    s_Dab[w][e] = D[a] + Db;
                    s_a[w][e] = a;
                    nu = (np + TRI_UNIT - 1) / TRI_UNIT;
                }
            }
            int inc = nu;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, inc, o);
                if (lane >= o) inc += y;
            }
            s_ex[w][e] = U + inc - nu;
            U += __shfl_sync(FULL, inc, 31);
        }
        __syncwarp();
        int cur_a = -1, hit_a = 0;
        int64_t acc_a = 0;
        int i = -1, kend = 0, exi = 0, b = 0, Db = 0, Dab = 0, ai = 0;
        int2 bpd = make_int2(0, 0);
        for (int t = lane; t < U; t += 32) {
            // the warp edge owning unit t: the last i with s_ex[i] <= t (s_ex is
            // non-decreasing; i + step <= EW - 1 at every step)
            int ni = 0;
#pragma unroll
            for (int step = EW / 2; step > 0; step >>= 1)
                if (s_ex[w][ni + step] <= t) ni += step;
            if (ni != i) {
                i = ni;
                kend = s_kend[w][i];
                exi = s_ex[w][i];
                b = s_b[w][i];
                Db = s_Db[w][i];
                bpd = s_bpd[w][i];
                Dab = s_Dab[w][i];
                ai = s_a[w][i];
            }
            const int64_t j0 = K0 + i + 1 + TRI_UNIT * (t - exi);
            const int jn = (int)min((int64_t)TRI_UNIT, kend - j0);
            int c[TRI_UNIT], Dc[TRI_UNIT];
            int2 rc[TRI_UNIT];
#pragma unroll
            for (int q = 0; q < TRI_UNIT; ++q) {
                if (q < jn) {
                    c[q] = __ldg(out_col + j0 + q);
                    Dc[q] = __ldg(out_D + j0 + q);
                    rc[q] = __ldg(out_pd + j0 + q);
                }
            }
            Probe pr[TRI_UNIT];
            int4 x[TRI_UNIT], y[TRI_UNIT];
#pragma unroll
            for (int q = 0; q < TRI_UNIT; ++q) {
                if (q < jn) {
                    const bool b_low = rank_less(Db, b, Dc[q], c[q]);
                    pr[q] = probe_of(out_col, out_hash, b_low ? bpd : rc[q], b_low ? c[q] : b);
                    pr[q].info |= (unsigned)b_low << 10;
                    x[q] = __ldg(pr[q].p0);
                    y[q] = __ldg(pr[q].p0 + pr[q].d1);
                }
            }
            int hits = 0;
            int64_t gsum = 0;
#pragma unroll
            for (int q = 0; q < TRI_UNIT; ++q) {
                if (q < jn) {
                    const bool b_low = (pr[q].info >> 10) & 1u;
                    if (probe_done(pr[q], x[q], y[q], out_col, out_hash, b_low ? bpd : rc[q], b_low ? c[q] : b)) {
                        const int64_t g = __ldg(tq + Dab + Dc[q]);
                        credit_tri(qacc, tcnt, c[q], g, 1);
                        gsum += g;
                        ++hits;
                    }
                }
            }
            if (hits) {
                credit_tri(qacc, tcnt, b, gsum, hits);
                if (ai != cur_a) {
                    if (hit_a) credit_tri(qacc, tcnt, cur_a, acc_a, hit_a);
                    cur_a = ai;
                    acc_a = 0;
                    hit_a = 0;
                }
                acc_a += gsum;
                hit_a += hits;
            }
        }
        if (hit_a) credit_tri(qacc, tcnt, cur_a, acc_a, hit_a);
        __syncwarp();
    }
}

static inline unsigned grid_of(int64_t work, int per_block, int64_t cap) {
    int64_t g = (work + per_block - 1) / per_block;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

int launch_tri_pairs(const Scratch &s, int32_t n, int64_t m, const Tune &t, cudaStream_t st,
                     const int32_t *owner_range) {
    const unsigned grid = grid_of(m / 2, TRI_WARPS * 32, (int64_t)t.num_sms * 16);
    if (t.tri_variant == 1)
        k_tri_pairs<4, 3, 32><<<grid, TRI_WARPS * 32, 0, st>>>(s.out_ptr, s.out_col, s.out_D, s.out_pd, s.out_src,
                                                            s.out_hash, s.outdeg, s.D, n, owner_range, s.tq, s.qacc,
                                                            s.tcnt, s.counters);
    else
        k_tri_pairs<2, 4, 64><<<grid, TRI_WARPS * 32, 0, st>>>(s.out_ptr, s.out_col, s.out_D, s.out_pd, s.out_src,
                                                            s.out_hash, s.outdeg, s.D, n, owner_range, s.tq, s.qacc,
                                                            s.tcnt, s.counters);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
