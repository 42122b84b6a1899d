// Triangle pass of libef (Algorithm 1, Phase 2: the "i in Adj(j)" test).
//
// The wedge pass credits every cluster with its open degree; clusters whose
// ends are adjacent (triangles) need d - 2 instead.  Edges are oriented from
// lower to higher (degree, id); each triangle {a, b, c} with a < b < c in
// that order is found once, by owner a, as c in N+(a) and c in N+(b) for
// b in N+(a).  Its three nodes each hold 4 credits of degree sum-6 that the
// wedge pass counted at sum-4 (sum = D_a + D_b + D_c), so each receives
// g = f(sum-6) - f(sum-4) here (times 4 in the finalize pass) and one
// triangle count.
//
// Credits to b and c are written to the slot of a in their rows (out_rslot),
// credits to a to tri_own[a].  The warp kernel keeps per-out-neighbour sums
// in shared memory and stores each slot once; the CTA kernel (owners with
// more than TRI_WARP_CAP out-neighbours) tiles N+(a) through shared memory
// and adds into pre-zeroed slots with global atomics (those slots belong to
// owner a alone, so the atomics are uncontended).
#include "ef_internal.cuh"

namespace ef {

constexpr int TRI_WARPS = 8;

__global__ void __launch_bounds__(TRI_WARPS * 32) k_tri_warp(
    const int32_t *__restrict__ out_ptr, const int32_t *__restrict__ out_col, const int32_t *__restrict__ out_D,
    const int32_t *__restrict__ out_rslot, const int32_t *__restrict__ D, const int32_t *__restrict__ list,
    const int32_t *__restrict__ cnt, const double *__restrict__ ftab, double *__restrict__ slotC,
    int32_t *__restrict__ slotT, double *__restrict__ tri_own, int64_t *__restrict__ t_own) {
    __shared__ int32_t s_id[TRI_WARPS][TRI_WARP_CAP];
    __shared__ int32_t s_d[TRI_WARPS][TRI_WARP_CAP];
    __shared__ double s_c[TRI_WARPS][TRI_WARP_CAP];
    __shared__ int32_t s_t[TRI_WARPS][TRI_WARP_CAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t *ids = s_id[w], *ds = s_d[w], *ts = s_t[w];
    double *cs = s_c[w];
    const int count = cnt[BIN_TW];
    const int64_t nwarps = (int64_t)gridDim.x * TRI_WARPS;
    for (int64_t oi = (int64_t)blockIdx.x * TRI_WARPS + w; oi < count; oi += nwarps) {
        const int a = list[oi];
        const int Da = D[a];
        const int s0 = out_ptr[a];
        const int p = out_ptr[a + 1] - s0;   // 2 <= p <= TRI_WARP_CAP
        for (int i = lane; i < p; i += 32) {
            ids[i] = out_col[s0 + i];
            ds[i] = out_D[s0 + i];
            cs[i] = 0.0;
            ts[i] = 0;
        }
        __syncwarp();
        double own = 0.0;
        int own_t = 0;
        for (int ib = 0; ib < p; ++ib) {   // N+(a) is in id order, so every b is scanned
            const int b = ids[ib];
            const int Db = ds[ib];
            const int q0 = out_ptr[b];
            const int q = out_ptr[b + 1] - q0;
            double bacc = 0.0;
            int bt = 0;
            for (int jc = lane; jc < q; jc += 32) {
                const int c = out_col[q0 + jc];
                const int pos = lower_bound_i32(ids, p, c);
                if (pos < p && ids[pos] == c) {
                    const int sum = Da + Db + ds[pos];
                    const double g = __ldg(ftab + (sum - 6)) - __ldg(ftab + (sum - 4));
                    own += g;
                    ++own_t;
                    bacc += g;
                    ++bt;
                    cs[pos] += g;   // distinct c per (b, lane) -> distinct pos: no conflict
                    ts[pos] += 1;
                }
            }
            bacc = warp_sum(bacc);
            bt = warp_sum(bt);
            __syncwarp();
            if (lane == 0) {
                cs[ib] += bacc;
                ts[ib] += bt;
            }
            __syncwarp();
        }
        for (int i = lane; i < p; i += 32) {
            const int r = out_rslot[s0 + i];
            slotC[r] = cs[i];
            slotT[r] = ts[i];
        }
        own = warp_sum(own);
        own_t = warp_sum(own_t);
        if (lane == 0) {
            tri_own[a] = own;
            t_own[a] = own_t;
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(TRI_CTA_THREADS) k_tri_cta(
    const int32_t *__restrict__ out_ptr, const int32_t *__restrict__ out_col, const int32_t *__restrict__ out_D,
    const int32_t *__restrict__ out_rslot, const int32_t *__restrict__ D, const int32_t *__restrict__ list,
    int32_t *__restrict__ cnt, const double *__restrict__ ftab, double *__restrict__ slotC,
    int32_t *__restrict__ slotT, double *__restrict__ tri_own, int64_t *__restrict__ t_own) {
    extern __shared__ __align__(16) int32_t smem[];
    int32_t *ids = smem;
    int32_t *ds = smem + TRI_CTA_SMEM_CAP;
    __shared__ int s_owner;
    __shared__ double s_red[TRI_CTA_THREADS / 32];
    __shared__ long long s_redt[TRI_CTA_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int NW = TRI_CTA_THREADS / 32;
    const int count = cnt[BIN_TC];
    for (;;) {
        if (threadIdx.x == 0) s_owner = atomicAdd(cnt + CNT_TRICTA, 1);
        __syncthreads();
        const int oi = s_owner;
        if (oi >= count) break;
        const int a = list[oi];
        const int Da = D[a];
        const int s0 = out_ptr[a];
        const int p = out_ptr[a + 1] - s0;
        double own = 0.0;
        long long own_t = 0;
        for (int t0 = 0; t0 < p; t0 += TRI_CTA_SMEM_CAP) {
            const int tn = min(TRI_CTA_SMEM_CAP, p - t0);
            __syncthreads();
            for (int i = threadIdx.x; i < tn; i += TRI_CTA_THREADS) {
                ids[i] = out_col[s0 + t0 + i];
                ds[i] = out_D[s0 + t0 + i];
            }
            __syncthreads();
            for (int ib = w; ib < p; ib += NW) {
                const int b = out_col[s0 + ib];
                const int Db = out_D[s0 + ib];
                const int q0 = out_ptr[b];
                const int q = out_ptr[b + 1] - q0;
                double bacc = 0.0;
                int bt = 0;
                for (int jc = lane; jc < q; jc += 32) {
                    const int c = out_col[q0 + jc];
                    const int pos = lower_bound_i32(ids, tn, c);
                    if (pos < tn && ids[pos] == c) {
                        const int sum = Da + Db + ds[pos];
                        const double g = __ldg(ftab + (sum - 6)) - __ldg(ftab + (sum - 4));
                        own += g;
                        ++own_t;
                        bacc += g;
                        ++bt;
                        const int r = out_rslot[s0 + t0 + pos];
                        atomicAdd(slotC + r, g);
                        atomicAdd(slotT + r, 1);
                    }
                }
                bacc = warp_sum(bacc);
                bt = warp_sum(bt);
                if (lane == 0 && bt) {
                    const int r = out_rslot[s0 + ib];
                    atomicAdd(slotC + r, bacc);
                    atomicAdd(slotT + r, bt);
                }
            }
        }
        own = warp_sum(own);
        own_t = warp_sum(own_t);
        if (lane == 0) {
            s_red[w] = own;
            s_redt[w] = own_t;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            double v = threadIdx.x < NW ? s_red[threadIdx.x] : 0.0;
            long long vt = threadIdx.x < NW ? s_redt[threadIdx.x] : 0;
            v = warp_sum(v);
            vt = warp_sum(vt);
            if (threadIdx.x == 0) {
                tri_own[a] = v;
                t_own[a] = vt;
            }
        }
    }
}

size_t tri_cta_grid(int num_sms) { return (size_t)num_sms * 2; }

int launch_triangles(const Scratch &s, int32_t n, int num_sms, cudaStream_t st) {
    const int32_t *tw = s.bins + (size_t)BIN_TW * n;
    const int32_t *tc = s.bins + (size_t)BIN_TC * n;
    int64_t g = ((int64_t)n + TRI_WARPS - 1) / TRI_WARPS;
    unsigned grid = (unsigned)(g < 1 ? 1 : (g > num_sms * 16 ? num_sms * 16 : g));
    k_tri_warp<<<grid, TRI_WARPS * 32, 0, st>>>(s.out_ptr, s.out_col, s.out_D, s.out_rslot, s.D, tw, s.counters,
                                                s.ftab, s.slotC, s.slotT, s.tri_own, s.t_own);
    size_t smem = (size_t)TRI_CTA_SMEM_CAP * 2 * sizeof(int32_t);
    k_tri_cta<<<(unsigned)tri_cta_grid(num_sms), TRI_CTA_THREADS, smem, st>>>(
        s.out_ptr, s.out_col, s.out_D, s.out_rslot, s.D, tc, s.counters, s.ftab, s.slotC, s.slotT, s.tri_own,
        s.t_own);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
