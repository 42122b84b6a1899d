// Triangle pass of libef (Algorithm 1, Phase 2: the "i in Adj(j)" test).
//
// The wedge pass credits every cluster with its open degree; clusters whose
// ends are adjacent (triangles) need d - 2 instead.  Edges are oriented from
// lower to higher (degree, id); each triangle {a, b, c} with a < b < c in
// that order is found exactly once, on the oriented edge a -> b, as an
// element c of N+(a) and N+(b).  Its three nodes each hold 4 credits of
// degree sum-6 that the wedge pass counted at sum-4 (sum = D_a + D_b + D_c),
// so each receives g = 4 (f(sum-6) - f(sum-4)) and one triangle count.
//
// One thread per oriented edge a -> b merges the two id-sorted out-lists
// (the whole oriented CSR is a few tens of MB and stays in L2).  Credits go
// where the wedge pass put a's credits to b and c -- the slot of a in their
// rows -- and a's own to Ccenter[a].  A hit is rare (in the power-law
// workload 2.7M of 20.6M oriented edges close a triangle), so credits to c
// use uncontended global atomics; credits to a and b are summed per thread
// and added once.
#include "ef_internal.cuh"

#include <type_traits>

namespace ef {

template <bool F64>
__global__ void __launch_bounds__(256) k_tri_edges(
    const int32_t *__restrict__ out_ptr, const int32_t *__restrict__ out_col, const int32_t *__restrict__ out_D,
    const int32_t *__restrict__ out_rslot, const int32_t *__restrict__ out_src, const int32_t *__restrict__ D,
    int32_t n, const double *__restrict__ ftab, void *__restrict__ slot_, int32_t *__restrict__ slotT,
    double *__restrict__ Ccenter, int64_t *__restrict__ t_own) {
    using Acc = typename std::conditional<F64, double, float>::type;
    Acc *slot = reinterpret_cast<Acc *>(slot_);
    const int64_t total = out_ptr[n];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int a = out_src[k];
        const int b = out_col[k];
        int x = out_ptr[a], xe = out_ptr[a + 1];
        int y = out_ptr[b], ye = out_ptr[b + 1];
        if (x >= xe || y >= ye) continue;
        const int Dab = D[a] + out_D[k];
        double acc = 0.0;
        int hits = 0;
        int va = out_col[x], vb = out_col[y];
        for (;;) {
            if (va < vb) {
                if (++x >= xe) break;
                va = out_col[x];
            } else if (va > vb) {
                if (++y >= ye) break;
                vb = out_col[y];
            } else {
                const int sum = Dab + out_D[x];
                const double g = 4.0 * (__ldg(ftab + (sum - 6)) - __ldg(ftab + (sum - 4)));
                const int rc = out_rslot[x];
                atomicAdd(slot + rc, (Acc)g);
                atomicAdd(slotT + rc, 1);
                acc += g;
                ++hits;
                if (++x >= xe || ++y >= ye) break;
                va = out_col[x];
                vb = out_col[y];
            }
        }
        if (hits) {
            const int rb = out_rslot[k];
            atomicAdd(slot + rb, (Acc)acc);
            atomicAdd(slotT + rb, hits);
            atomicAdd(Ccenter + a, acc);
            atomicAdd((unsigned long long *)(t_own + a), (unsigned long long)hits);
        }
    }
}

int launch_triangles(const Scratch &s, int precision, int32_t n, int64_t m, int num_sms, cudaStream_t st) {
    int64_t g = (m / 2 + 255) / 256;
    unsigned grid = (unsigned)(g < 1 ? 1 : (g > (int64_t)num_sms * 64 ? (int64_t)num_sms * 64 : g));
    if (precision == EF_PREC_FP64)
        k_tri_edges<true><<<grid, 256, 0, st>>>(s.out_ptr, s.out_col, s.out_D, s.out_rslot, s.out_src, s.D, n, s.ftab,
                                                s.slotR, s.slotT, s.Ccenter, s.t_own);
    else
        k_tri_edges<false><<<grid, 256, 0, st>>>(s.out_ptr, s.out_col, s.out_D, s.out_rslot, s.out_src, s.D, n,
                                                 s.ftab, s.slotR, s.slotT, s.Ccenter, s.t_own);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
