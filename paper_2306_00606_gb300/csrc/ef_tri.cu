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
// lower-ranked one's out-list (binary search; the oriented CSR is a few tens
// of MB and stays in L2).  That is sum_a C(|N+(a)|, 2) independent tests --
// 1.1e8 on the 4M-node power-law workload, against 1.15e9 dependent steps
// for merging the two out-lists of every edge.  A warp takes 32 consecutive
// oriented edges and spreads all their pairs evenly over its lanes.
//
// The pass is integer-only: g comes from a table in fixed point (units of
// 2^-F, F chosen per call from the maximum degree), so the sums are exact and
// independent of the order of the atomics, and no FP64 instruction (one lane
// per clock per SM sub-partition on this GPU) sits in a divergent branch.
// Corrections and counts go to per-node accumulators (qacc, tcnt) by L2
// reductions: c's at once, a's and b's merged per lane over consecutive hits
// (a lane's pairs share a, and often b).
#include "ef_internal.cuh"

namespace ef {

constexpr int TRI_WARPS = 8;

__device__ __forceinline__ void credit_tri(int64_t *qacc, int64_t *tcnt, int v, int64_t q, int cnt) {
    atomicAdd((unsigned long long *)(qacc + v), (unsigned long long)q);
    atomicAdd((unsigned long long *)(tcnt + v), (unsigned long long)cnt);
}

__global__ void __launch_bounds__(TRI_WARPS * 32) k_tri_pairs(
    const int32_t *__restrict__ out_ptr, const int32_t *__restrict__ out_col, const int32_t *__restrict__ out_D,
    const int32_t *__restrict__ out_src, const int32_t *__restrict__ D, int32_t n, const int64_t *__restrict__ tq,
    int64_t *__restrict__ qacc, int64_t *__restrict__ tcnt) {
    __shared__ int s_ex[TRI_WARPS][32];   // exclusive prefix of pair counts
    __shared__ int s_k[TRI_WARPS][32], s_b[TRI_WARPS][32], s_Db[TRI_WARPS][32], s_bs[TRI_WARPS][32];
    __shared__ int s_be[TRI_WARPS][32], s_Dab[TRI_WARPS][32], s_a[TRI_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t total = out_ptr[n];
    const int64_t stride = (int64_t)gridDim.x * TRI_WARPS * 32;
    for (int64_t K0 = ((int64_t)blockIdx.x * TRI_WARPS + w) * 32; K0 < total; K0 += stride) {
        const int64_t k = K0 + lane;
        int np = 0;
        if (k < total) {
            const int a = out_src[k];
            const int kend = out_ptr[a + 1];
            np = kend - (int)k - 1;
            if (np > 0) {
                const int b = out_col[k];
                const int Db = out_D[k];
                s_k[w][lane] = (int)k;
                s_b[w][lane] = b;
                s_Db[w][lane] = Db;
                s_bs[w][lane] = out_ptr[b];
                s_be[w][lane] = out_ptr[b + 1];
                s_Dab[w][lane] = D[a] + Db;
                s_a[w][lane] = a;
            } else {
                np = 0;
            }
        }
        int inc = np;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        s_ex[w][lane] = inc - np;
        const int P = __shfl_sync(FULL, inc, 31);
        __syncwarp();
        int cur_i = -1, cur_a = -1, hit_b = 0, hit_a = 0;
        int64_t acc_b = 0, acc_a = 0;
        int i = -1, ki = 0, exi = 0, b = 0, Db = 0, bs = 0, be = 0, Dab = 0, ai = 0;
        for (int t = lane; t < P; t += 32) {
            // the warp edge owning pair t: the last i with s_ex[i] <= t (s_ex is
            // non-decreasing; i + step <= 31 at every step)
            int ni = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (s_ex[w][ni + step] <= t) ni += step;
            if (ni != i) {
                i = ni;
                ki = s_k[w][i];
                exi = s_ex[w][i];
                b = s_b[w][i];
                Db = s_Db[w][i];
                bs = s_bs[w][i];
                be = s_be[w][i];
                Dab = s_Dab[w][i];
                ai = s_a[w][i];
            }
            const int j = ki + 1 + (t - exi);
            const int c = out_col[j];
            const int Dc = out_D[j];
            const bool b_low = rank_less(Db, b, Dc, c);
            const int ls = b_low ? bs : out_ptr[c];
            const int le = b_low ? be : out_ptr[c + 1];
            const int key = b_low ? c : b;
            const int pos = ls + lower_bound_i32(out_col + ls, le - ls, key);
            if (pos < le && out_col[pos] == key) {
                const int64_t q = tq[Dab + Dc];
                credit_tri(qacc, tcnt, c, q, 1);
                if (i != cur_i) {
                    if (hit_b) credit_tri(qacc, tcnt, s_b[w][cur_i], acc_b, hit_b);
                    cur_i = i;
                    acc_b = 0;
                    hit_b = 0;
                }
                acc_b += q;
                ++hit_b;
                if (ai != cur_a) {
                    if (hit_a) credit_tri(qacc, tcnt, cur_a, acc_a, hit_a);
                    cur_a = ai;
                    acc_a = 0;
                    hit_a = 0;
                }
                acc_a += q;
                ++hit_a;
            }
        }
        if (hit_b) credit_tri(qacc, tcnt, s_b[w][cur_i], acc_b, hit_b);
        if (hit_a) credit_tri(qacc, tcnt, cur_a, acc_a, hit_a);
        __syncwarp();
    }
}

int launch_triangles(const Scratch &s, int32_t n, int64_t m, int num_sms, cudaStream_t st) {
    int64_t g = (m / 2 + TRI_WARPS * 32 - 1) / (TRI_WARPS * 32);
    unsigned grid = (unsigned)(g < 1 ? 1 : (g > (int64_t)num_sms * 16 ? (int64_t)num_sms * 16 : g));
    k_tri_pairs<<<grid, TRI_WARPS * 32, 0, st>>>(s.out_ptr, s.out_col, s.out_D, s.out_src, s.D, n, s.tq, s.qacc,
                                                 s.tcnt);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
