// Internal declarations of libef: device helpers, scratch layout, kernels.
//
// Notation follows the paper ("Scaling Expected Force", Algorithm 1):
//   D_x      degree of node x, N(x) its sorted neighbour row;
//   a cluster (i, u, j) has middle node u and ends i < j in N(u); its open
//   degree is d0 = D_u + D_i + D_j - 4 and its degree is d = d0 - 2 when
//   i and j are adjacent (a triangle), d = d0 otherwise;
//   credits: 2 to the middle node, 1 to each end.
//   f(d) = d ln d; per node S = sum credit*d, T = sum credit*f(d).
//
// The wedge pass credits every cluster with its open degree d0.  The
// triangle pass lists each triangle {a, b, c} once and corrects its three
// wedges: each of a, b, c holds 4 credits of that triangle's clusters (2 as
// middle, 1 + 1 as an end), all of degree sum - 6 instead of sum - 4, where
// sum = D_a + D_b + D_c.  So each node of the triangle gets
// 4 * (f(sum-6) - f(sum-4)) added to T and -8 added to S.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ef.h"

namespace ef {

constexpr unsigned FULL = 0xffffffffu;

// Error bits set on the device by the validation kernels.
enum : int {
    ERRB_ROWPTR = 1,    // row_ptr not monotone, row_ptr[0] != 0 or row_ptr[n] != m
    ERRB_RANGE = 2,     // a column index outside [0, n)
    ERRB_SELFLOOP = 4,  // v in N(v)
    ERRB_UNSORTED = 8,  // a row not strictly ascending (includes duplicates)
    ERRB_ASYM = 16,     // x in N(u) but u not in N(x)
};

// Work bins.  Middle nodes are binned by degree for the wedge pass; triangle
// owners (nodes with >= 2 out-neighbours in degree order) by out-degree.
enum : int {
    BIN_S4 = 0,   // 1 <= D <= 4   (8 middle nodes per warp)
    BIN_S8,       // 5..8          (4 per warp)
    BIN_S16,      // 9..16         (2 per warp)
    BIN_S32,      // 17..32        (1 per warp)
    BIN_BIG,      // D > 32        (CTA work items)
    BIN_TW,       // 2 <= out-degree <= TRI_WARP_CAP (warp per owner)
    BIN_TC,       // out-degree > TRI_WARP_CAP (CTA per owner)
    NUM_BINS
};

constexpr int SMALL_MAX = 32;
constexpr int TRI_WARP_CAP = 128;
constexpr int BIG_ROWS = 256;          // rows (neighbours) per big work item = threads per CTA
constexpr int BIG_TILE = 4096;         // neighbour degrees staged in shared memory per tile
constexpr int TRI_CTA_THREADS = 512;
constexpr int TRI_CTA_SMEM_CAP = 6000; // out-neighbours per shared-memory tile of the CTA kernel (48000 B)

// Scratch carved from one device allocation per call (sizes depend on n, m).
struct Scratch {
    int32_t *D;          // n      degrees
    int64_t *sig1;       // n      sum of neighbour degrees
    int64_t *sig2;       // n      sum of squared neighbour degrees
    int64_t *omega;      // n      sum of neighbours' sig1
    int32_t *outdeg;     // n      out-degree in degree order
    int32_t *out_ptr;    // n+1    oriented CSR offsets
    int32_t *out_col;    // m/2+1  oriented neighbour ids (ascending id within a row)
    int32_t *out_D;      // m/2+1  their degrees
    int32_t *out_rslot;  // m/2+1  slot of the reverse entry (position of the owner in the neighbour's row)
    int32_t *rev;        // m      rev[e] = position of u in N(x) for e = (u -> x)
    void    *slotR;      // m      open-degree credit to the row owner from the column node as middle (float or double)
    double  *slotC;      // m      triangle correction to the row owner found by the column node as owner
    int32_t *slotT;      // m      triangle count credited the same way
    double  *Ccenter;    // n      middle-node credit sum (2 * sum over pairs of f(d0))
    double  *tri_own;    // n      triangle corrections found as owner (sum of f(s-6)-f(s-4))
    int64_t *t_own;      // n      triangles found as owner
    int32_t *bins;       // NUM_BINS * n   work lists
    int32_t *counters;   // 64 ints: [0..NUM_BINS) bin counts, [16] error word, [17] max degree,
                         //          [18] big item counter, [19] triangle CTA counter, [20] timeout flag
    int32_t *big_chunks; // n+1    work items per big middle node, then its exclusive scan
    double  *big_partial;// m/BIG_ROWS + n + 1  per-item middle-node partial sums
    int32_t *scan_tmp;   // scan block sums
    double  *ftab;       // 3*maxdeg+1 (capacity): f(d) = d ln d in FP64
    int32_t *tri_gl;     // global overflow arrays for huge triangle owners
    int64_t tri_gl_cap;  // entries per CTA
};

enum : int { CNT_ERR = 16, CNT_MAXDEG = 17, CNT_BIGITEM = 18, CNT_TRICTA = 19 };

// ----------------------------------------------------------------- helpers
__device__ __forceinline__ bool rank_less(int32_t Dx, int32_t x, int32_t Dy, int32_t y) {
    // degree order used to orient edges for triangle listing: (degree, id)
    return Dx < Dy || (Dx == Dy && x < y);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// lower_bound over a sorted int32 array (generic address space)
__device__ __forceinline__ int lower_bound_i32(const int32_t *a, int len, int32_t key) {
    int lo = 0, hi = len;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Kahan-compensated FP32 accumulation (compensation kept in c).
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

// d * log2(d) for integral d >= 1 held in a float (MUFU lg2).
__device__ __forceinline__ float dlog2d(float d) { return d * __log2f(d); }

constexpr double LN2 = 0.69314718055994530942;

}  // namespace ef

// ------------------------------------------------------------ launchers
namespace ef {
int launch_prep_a(const int32_t *rp, const int32_t *ci, int32_t n, int64_t m, const Scratch &s, cudaStream_t st);
int launch_prep_b(const int32_t *rp, const int32_t *ci, int32_t n, int64_t m, const Scratch &s, cudaStream_t st);
int launch_scan(const int32_t *in, int32_t *out, int32_t n, int32_t *tmp, cudaStream_t st);
int launch_ftab(double *ftab, const int32_t *maxdeg_dev, int64_t cap, cudaStream_t st);
int launch_wedge_small(const int32_t *rp, const int32_t *ci, const Scratch &s, int precision, int32_t n,
                       cudaStream_t st);
int launch_wedge_big(const int32_t *rp, const int32_t *ci, const Scratch &s, int precision, int32_t n,
                     int64_t m, int num_sms, cudaStream_t st);
int launch_triangles(const Scratch &s, int32_t n, int num_sms, cudaStream_t st);
int launch_finalize(const int32_t *rp, const int32_t *ci, const Scratch &s, int precision, int32_t n,
                    const ef_outputs &out, cudaStream_t st);
size_t tri_cta_grid(int num_sms);
}  // namespace ef
