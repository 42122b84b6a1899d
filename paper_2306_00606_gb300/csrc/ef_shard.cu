// Shards of the per-node sums (Eq. 1 decomposed; Algorithm 1's cluster loop
// split between independent workers).
//
// EF(v) = ln S_v - T_v / S_v needs, besides closed forms in v's degree sums
// (written by the shard that owns v), three per-node sums over v's clusters:
//   T_v   sum of d ln d with open degrees (wedge pass),
//   q_v   triangle corrections in fixed point 2^-F (triangle pass),
//   t_v   triangles at v (triangle pass).
// Each wedge credits its three nodes from its middle node; each triangle
// credits its three nodes from its lowest-ranked node in the (degree, id)
// order.  Shard r of R owns the nodes [lo, hi) cut at adjacency entry r m / R
// and takes the wedges whose middle node, and the triangles whose
// lowest-ranked node, lies in its range.  (The wedge kernels here spend O(D)
// per middle node after the degree-class compression, and a node of
// out-degree p opens C(p, 2) pair tests with p <= D, so equal shares of
// row_ptr are near-equal shares of both.)  Every wedge and every triangle is
// counted by exactly one shard, so the element-wise sums of the shards'
// partials are the whole graph's T, q, t: q and t exactly, T up to the order
// of its FP64 additions.  F depends on the maximum degree only, so every
// shard and the finalize use the same one.
#include "ef_internal.cuh"

namespace ef {

// range = [lo, hi): lo is the first row starting at or after entry
// shard m / R (0 for the first shard, n after the last).
__global__ void k_shard_range(const int32_t *__restrict__ rp, int32_t n, int64_t m, int32_t shard, int32_t nshards,
                              int32_t *__restrict__ range) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    auto node_cut = [&](int32_t r) -> int32_t {
        if (r <= 0) return 0;
        if (r >= nshards) return n;
        return lower_bound_i32(rp, n + 1, (int32_t)(m * r / nshards));
    };
    range[0] = node_cut(shard);
    range[1] = node_cut(shard + 1);
}

__global__ void k_mark_range(const int32_t *__restrict__ range, int32_t n, int32_t *__restrict__ mark) {
    const int lo = range[0], hi = range[1];
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        mark[v] = v >= lo && v < hi;
}

// The shard's partials of every node: its middle-node credit (in range), the
// end credits its middle nodes pushed, its triangles' corrections, and for
// its own nodes the closed forms (Algorithm 1's credited counts and degree
// sums at open degrees)
//   N_v      = D(D-2) + sigma1,
//   S_open_v = D(D-1)(D-4) + 2(D-1) sigma1 + sigma2 - sigma1
//              + (D-4)(sigma1 - D) + omega - D^2.
template <bool F64>
__global__ void __launch_bounds__(256) k_shard_out(const int32_t *__restrict__ range, const Scratch s, int32_t n,
                                                   ef_partials p) {
    const int lo = range[0], hi = range[1];
    const AccT<F64> *cc = reinterpret_cast<const AccT<F64> *>(s.Ccenter);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const bool own = v >= lo && v < hi;
        const int64_t d = s.D[v];
        const double c = own && d >= 2 ? (double)cc[v] : 0.0;
        p.t[v] = c + s.Tacc[v];
        p.q[v] = s.qacc[v];
        p.triangles[v] = s.tcnt[v];
        int64_t N = 0, S = 0;
        if (own) {
            const int64_t s1 = s.sig1[v], s2 = s.sig2[v], om = s.omega[v];
            N = d * (d - 2) + s1;
            S = d * (d - 1) * (d - 4) + 2 * (d - 1) * s1 + s2 - s1 + (d - 4) * (s1 - d) + om - d * d;
        }
        p.n_clusters[v] = N;
        p.s_open[v] = S;
    }
}

static inline unsigned grid_n(int32_t n, const Tune &t) {
    int64_t g = ((int64_t)n + 255) / 256;
    const int64_t cap = (int64_t)t.num_sms * 32;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

int launch_shard_range(const int32_t *rp, int32_t n, int64_t m, int32_t shard, int32_t nshards, int32_t *range,
                       cudaStream_t st) {
    k_shard_range<<<1, 32, 0, st>>>(rp, n, m, shard, nshards, range);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_mark_range(const int32_t *range, int32_t n, int32_t *mark, const Tune &t, cudaStream_t st) {
    k_mark_range<<<grid_n(n, t), 256, 0, st>>>(range, n, mark);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_shard_out(const int32_t *range, const Scratch &s, int precision, int32_t n, const ef_partials &out,
                     const Tune &t, cudaStream_t st) {
    if (precision == EF_PREC_FP64)
        k_shard_out<true><<<grid_n(n, t), 256, 0, st>>>(range, s, n, out);
    else
        k_shard_out<false><<<grid_n(n, t), 256, 0, st>>>(range, s, n, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
