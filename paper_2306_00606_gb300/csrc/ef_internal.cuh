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
//
// Per-node accumulators (a few tens of MB, resident in L2) collect what
// nodes send each other: the middle node u reduces its own credit with warp
// shuffles and stores it once (Ccenter[u]); its open-degree credit to each
// end x, R_u(x), is added to Tacc[x] with a fire-and-forget L2 reduction (one
// per CSR entry; a node receives its D_x of them spread over the whole pass,
// so they do not contend); triangle corrections go to qacc (exact fixed
// point) and tcnt the same way.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

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
    ERRB_CROSS = 32,    // batched input: an entry outside its row's graph
    ERRB_NODE = 64,     // a requested node id outside [0, n)
    ERRB_SIR_ARG = 128, // SIR: an index case outside [0, n) or immune, or an immune-set index out of range
    ERRB_DEGREE = 256,  // device-side check: the maximum degree is above EF_MAX_DEGREE
};

// Work bins (each a list of node ids of capacity n), filled from the degrees.
enum : int {
    BIN_S4 = 0,    // 1 <= D <= 4   middle nodes, 8 per warp
    BIN_S8,        // 5..8          4 per warp
    BIN_S16,       // 9..16         2 per warp
    BIN_S32,       // 17..32        1 per warp
    BIN_BIG,       // D > 32        (direct wedge kernel)
    BIN_MID,       // 32 < D < hub_min (<= MID_MAX)   degree-class wedge kernel, one warp each
    BIN_HUB0,      // D >= hub_min, bucket floor(log2 D) - 9 clamped to [0, NUM_HUB_BUCKETS-1]
    BIN_HUB_LAST = BIN_HUB0 + 6,
    NUM_BINS
};
constexpr int NUM_HUB_BUCKETS = BIN_HUB_LAST - BIN_HUB0 + 1;

constexpr int SMALL_MAX = 32;
constexpr int MID_MAX = 512;
constexpr int MID_HIST = 256;          // dense degree histogram of the warp-level class kernel
constexpr int HUB_HIST = 2048;         // dense degree histogram of the CTA-level class kernel
constexpr int HUB_THREADS = 512;
constexpr int HUB_SMEM_K = 4096;       // classes held in shared memory by the CTA kernel
constexpr int BIG_ROWS = 256;          // rows per work item of the direct big-node kernel
constexpr int BIG_TILE = 4096;         // neighbour degrees staged per tile by the direct kernel
constexpr int ROW_CTA = 512;           // threads of the per-hub-row kernels
constexpr int SHORT_MAX = 5;           // out-lists longer than this get a hash table for the triangle pass

// Triangle corrections are integers in units of 2^-F (the pass adds only
// integers: exact and independent of the order of the atomics).  F is chosen
// per call from the maximum degree as the largest value, at most 52, for
// which C(maxdeg, 2) triangles of the largest |g| cannot overflow int64
// (F = 52 on small graphs, 27 on the 4M-node power-law workload).
constexpr int TRI_FRAC_MAX = 52;

// Precision-dependent accumulator type: double (FP64) or float (FP32C).
template <bool F64>
using AccT = typename std::conditional<F64, double, float>::type;

// Launch parameters an autotuner may change (ef_tuning in ef.h); every
// choice gives the same results.
struct Tune {
    int row_thread_max = SMALL_MAX;   // row passes: rows of degree <= this take one thread each
    int hub_min = MID_MAX + 1;        // rows / middle nodes of degree >= this take a CTA (33..MID_MAX+1)
    int tri_variant = 0;              // pair-test kernel: 0 two candidates per lane step, 1 four
    int grid_per_sm = 64;             // blocks per SM of the grid-stride row passes
    int layout = 0;                   // oriented CSR: 0 automatic, 1 node order, 2 degree-bin order
    int num_sms = 0;
    unsigned grid(int64_t work, int per_block) const {
        int64_t g = (work + per_block - 1) / per_block;
        const int64_t cap = (int64_t)num_sms * grid_per_sm;
        return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
    }
};

// Scratch carved from one device allocation per call (sizes depend on n, m).
struct Scratch {
    int32_t *D;          // n      degrees
    int64_t *sig1;       // n      sum of neighbour degrees
    int64_t *sig2;       // n      sum of squared neighbour degrees
    int64_t *omega;      // n      sum of the neighbours' sigma1
    int32_t *outdeg;     // n      out-degree in (degree, id) order
    int32_t *out_ptr;    // n+1    oriented CSR offsets (a list runs from out_ptr[v] for outdeg[v] entries;
                         //        out_ptr[n] = all entries); lists are stored in layout order
    int32_t *lay_node;   // n      layout order: the work bins concatenated (degree classes)
    int32_t *lay_ptr;    // n+1    out-degrees in layout order, then their scan
    int4    *info;       // n      {D, sigma1, out_ptr, out_ptr next} per node, for the orientation
    int32_t *out_col;    // m+8    oriented neighbour ids (ascending id within a row)
    int32_t *out_D;      // m+1    their degrees
    int2    *out_pd;     // m+1    probe descriptors of their own out-lists (probe_desc)
    int32_t *out_hash;   // m+8    hash tables of the out-lists longer than SHORT_MAX
    int32_t *out_src;    // m+1    owner of each oriented edge
    double  *Tacc;       // n      open-degree credits received as an end (FP64 reductions)
    void    *Ccenter;    // n      middle-node credit (AccT<F64>, 8 bytes reserved per node)
    int64_t *qacc;       // n      triangle corrections, fixed point
    int64_t *tcnt;       // n      triangles
    int64_t *tq;         // 3*maxdeg+1 (capacity): 4 (f(s-6) - f(s-4)) * 2^F, rounded (F in counters)
    int32_t *bins;       // NUM_BINS * n   work lists
    int32_t *counters;   // NUM_COUNTERS ints: [0..NUM_BINS) bin counts, CNT_* below
    int32_t *big_chunks; // n+1    work items per big middle node (direct kernel), scanned in place
    double  *big_partial;// m/BIG_ROWS + n + 2  per-item middle-node partial sums (direct kernel)
    int32_t *scan_tmp;   // scan block sums (orientation)
    int32_t *scan_tmp2;  // scan block sums (direct kernel's items)
    float2  *ftab;       // 3*maxdeg+1 (capacity): f(d) = d ln d as an FP32 pair hi + lo (F2Sum)
    void    *hub_cls;    // m+n+2  class (degree, count) pairs of hubs with > HUB_SMEM_K classes
    void    *hub_q;      // m+n+2  their per-class credits
    int32_t *hub_cidx;   // m+1    class index of each neighbour of a hub (at the hub's row positions)
};

enum : int {
    CNT_ERR = 32,
    CNT_MAXDEG = 33,
    CNT_BIGITEM = 34,
    CNT_MIDITEM = 35,
    CNT_HUB = 36,
    CNT_TRIFRAC = 37,
    CNT_RANGE = 40,   // 40, 41: a shard's node range [lo, hi)
    CNT_SYM = 44,     // 44, 45: the symmetry sum (uint64, 8-byte aligned)
    CNT_BIGLO = 46,   // n - 1 - (smallest id of a node of degree > SMALL_MAX), if any
    CNT_BIGHI = 47,   // largest id of a node of degree > SMALL_MAX, if any
    CNT_GATE = 48,    // device-side check: the call's validation bits (0: part B runs), see gate_closed
    NUM_COUNTERS = 64
};

// Order of the oriented out-lists: degree-bin order (true) or node order,
// from t.layout, or in automatic mode (0) from where the nodes of degree >
// SMALL_MAX lie in a host copy of the counters after the degree pass (h;
// nullptr when none was read back): degree bins when they span more than
// half of the ids (their hot out-lists would be scattered in node order),
// node order when they are clustered or absent (lattices, BA and R-MAT
// graphs number their hubs close together).  Without counters: degree bins
// for one graph, node order for a batch.
inline bool bin_layout(const Tune &t, const int32_t *h, int32_t n, bool batched) {
    if (t.layout != 0) return t.layout == 2;
    if (!h) return !batched;
    if (h[BIN_BIG] == 0) return false;
    const int64_t lo = (int64_t)n - 1 - h[CNT_BIGLO], hi = h[CNT_BIGHI];
    return hi - lo > (int64_t)n / 2;
}

// Validation bits of a host copy of the counters after the row passes: the
// device's error word, and asymmetry when the symmetry sum is not 0.
inline int prep_error_bits(const int32_t *h) {
    uint64_t sym;
    memcpy(&sym, h + CNT_SYM, sizeof sym);
    return h[CNT_ERR] | (sym ? ERRB_ASYM : 0);
}

// Bytes of scratch for a graph (f tables excluded), and its layout when base != nullptr.
size_t carve_scratch(char *base, int32_t n, int64_t m, Scratch &s);
// Bytes from Tacc to the end of the counters: everything that must start at
// zero (Tacc, qacc, tcnt, counters), for one memset per call.
size_t accumulator_bytes(const Scratch &s);

// ----------------------------------------------------------------- helpers
// Device-side validation (ef_options.device_check): k_gate stores the call's
// validation bits in cnt[CNT_GATE] once the row passes are done, and every
// kernel after them returns at once when they are set, so nothing indexes by
// the column ids (or by anything derived from them) of a graph that failed.
// The word is 0 in every other mode: the counters start at zero each call,
// and the host refuses an invalid graph before part B.
__device__ __forceinline__ bool gate_closed(const int32_t *cnt) { return cnt[CNT_GATE] != 0; }

__device__ __forceinline__ bool rank_less(int32_t Dx, int32_t x, int32_t Dy, int32_t y) {
    // degree order used to orient edges for triangle listing: (degree, id)
    return Dx < Dy || (Dx == Dy && x < y);
}

// Symmetry check: every stored entry (v, x) adds
//   edge_print(v, x) = a_v b_x - a_x b_v   (mod 2^64)
// to one global sum, with a = a 32-bit mix of the node id (the MurmurHash3
// finaliser) and b = a * odd + c (mod 2^32), multiplied as 64-bit products.
// The term is antisymmetric, so in a symmetric CSR each entry's reverse
// cancels it and the sum is 0; the terms of entries without their reverse
// are pseudo-random 64-bit values that cancel only by accident (rows are
// strictly ascending, so no entry repeats).
struct NodeMix {
    uint32_t a, b;
};
__device__ __forceinline__ NodeMix node_mix(int32_t x) {
    uint32_t h = (uint32_t)x;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return NodeMix{h, h * 0x9E3779B1u + 0x7F4A7C15u};
}
__device__ __forceinline__ uint64_t edge_print(NodeMix v, NodeMix x) {
    return (uint64_t)v.a * x.b - (uint64_t)x.a * v.b;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Sum of a value over a group of G consecutive lanes (tree order).
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o, G);
    return v;
}

// lower_bound over a sorted int32 array (generic address space)
// ----------------------------------------------- out-list membership tables
// Table of the out-list [ls, le) of one node: slots [base, base + 4 nb) of
// out_hash, base = 2 ls rounded up to a multiple of 4 and 4 nb = 2 (le - ls)
// rounded down to one, so the tables of consecutive out-lists never overlap
// and every bucket is 16-byte aligned.  Only lists longer than SHORT_MAX have
// one, and only when it lies inside the array (always, for a symmetric CSR:
// the out-lists then hold m/2 entries in all).
__host__ __device__ __forceinline__ int64_t hash_slots(int64_t m) { return m + 8; }   // slots of out_hash

__device__ __forceinline__ bool out_table(int ls, int le, int64_t hash_cap, int64_t &base, int &nb) {
    const int p = le - ls;
    base = ((int64_t)2 * ls + 3) & ~(int64_t)3;
    nb = (2 * p) >> 2;
    return p > SHORT_MAX && base + 4 * (int64_t)nb <= hash_cap;
}

// Home bucket of key in a table of nb buckets of 4 slots.
__device__ __forceinline__ int bucket_of(int key, int nb) {
    const uint32_t h = (uint32_t)key * 0x9E3779B1u;
    return (int)(((uint64_t)h * (uint32_t)nb) >> 32);
}

// Insert key into a table (cleared to -1 beforehand) shared by several
// threads: linear probing over slots from the key's home bucket, by atomics.
__device__ __forceinline__ void table_insert_shared(int32_t *out_hash, int64_t base, int nb, int key) {
    const int cap = 4 * nb;
    int sl = 4 * bucket_of(key, nb);
    for (int tries = 0; tries < cap; ++tries) {
        const int prev = atomicCAS(out_hash + base + sl, -1, key);
        if (prev == -1 || prev == key) break;
        sl = sl + 1 == cap ? 0 : sl + 1;
    }
}

// Bits of the quad of entries [e0, e0 + 4) that lie in [ls, le).
__device__ __forceinline__ unsigned range_bits(int e0, int ls, int le) {
    const int lo = max(ls - e0, 0), hi = min(le - e0, 4);
    return hi > lo ? ((1u << hi) - 1u) & ~((1u << lo) - 1u) : 0u;
}

// Probe descriptor of the out-list [ls, le) (what the triangle pass needs to
// test membership in it, decided once per node instead of once per test):
//   kind 0, a list of at most SHORT_MAX entries: x = its first quad of
//     out_col, y = which entries of that quad (bits 0-3) and the next (4-7)
//     belong to it;
//   kind 1, a hashed list: x = its first bucket (quad) of out_hash, y = the
//     bucket count;
//   kind 2, a longer list without a table (malformed input only): x = ls,
//     y = le.
// The kind sits in bits 30-31 of y (counts and offsets stay below 2^30).
constexpr int DESC_KIND_SHIFT = 30;
constexpr int DESC_MASK = (1 << DESC_KIND_SHIFT) - 1;
__device__ __forceinline__ int2 probe_desc(int ls, int le, int64_t hash_cap) {
    int64_t hb;
    int nb;
    if (out_table(ls, le, hash_cap, hb, nb))
        return make_int2((int)(hb >> 2), (int)((unsigned)nb | 1u << DESC_KIND_SHIFT));
    if (le - ls > SHORT_MAX) return make_int2(ls, (int)((unsigned)le | 2u << DESC_KIND_SHIFT));
    const int q0 = ls >> 2;
    return make_int2(q0, (int)(range_bits(4 * q0, ls, le) | range_bits(4 * q0 + 4, ls, le) << 4));
}

__device__ __forceinline__ int lower_bound_i32(const int32_t *a, int len, int32_t key) {
    int lo = 0, hi = len;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Total number of hub rows (degree > MID_MAX) in the hub buckets.
__device__ __forceinline__ int hub_total(const int32_t *cnt) {
    int t = 0;
#pragma unroll
    for (int b = 0; b < NUM_HUB_BUCKETS; ++b) t += cnt[BIN_HUB0 + b];
    return t;
}

// The item-th hub row, largest degree bucket first (item < hub_total).
__device__ __forceinline__ int hub_row(const int32_t *bins, int32_t n, const int32_t *cnt, int item) {
    int b = NUM_HUB_BUCKETS - 1;
    while (item >= cnt[BIN_HUB0 + b]) item -= cnt[BIN_HUB0 + b--];
    return bins[(size_t)(BIN_HUB0 + b) * n + item];
}

// Kahan-compensated FP32 accumulation (compensation kept in c).
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Running sum in T: plain for double, Kahan-compensated for float.
template <typename T>
struct SumAcc {
    T s = 0, c = 0;
    __device__ __forceinline__ void add(T x) {
        if constexpr (sizeof(T) == 4) {
            kahan_add(s, c, x);
        } else {
            s += x;
        }
    }
    __device__ __forceinline__ T get() const { return s - c; }
};

// FP64-mode sums of f terms in FP32 pairs.  The f table holds each f(d) =
// d ln d (computed in FP64) as an unevaluated sum hi + lo of two floats
// (48 significant bits).  F2Sum adds terms c (hi + lo), c an integer below
// 2^24, to a running pair (sh, sl): c hi is split exactly into p + pe with
// an FMA, p goes into sh by an error-free two-sum whose error, pe and c lo
// collect in sl.  Every term here is >= 0, so over a chunk of at most
// F2_CHUNK terms each error is at most 2^-24 of the chunk's sum and sl's own
// rounding adds at most F2_CHUNK^2 2^-48 of it: below 2^-38 (3.6e-12)
// relative for chunks of 32, which the caller then adds up in FP64.  Each
// term costs about ten FP32 instructions instead of an FP64 FMA, which runs
// at a thirty-second of the FP32 rate on this GPU.
constexpr int F2_CHUNK = 32;
struct F2Sum {
    float sh = 0.f, sl = 0.f;
    __device__ __forceinline__ void add(float2 t, float c) {
        const float p = c * t.x;
        const float pe = fmaf(c, t.x, -p);   // c t.x - p, exactly
        const float s = sh + p;
        const float bp = s - sh;
        sl += ((sh - (s - bp)) + (p - bp)) + fmaf(c, t.y, pe);
        sh = s;
    }
    __device__ __forceinline__ void add(float2 t) {   // c = 1
        const float s = sh + t.x;
        const float bp = s - sh;
        sl += ((sh - (s - bp)) + (t.x - bp)) + t.y;
        sh = s;
    }
    __device__ __forceinline__ double value() const { return (double)sh + (double)sl; }
};
__device__ __forceinline__ double f2_value(float2 t) { return (double)t.x + (double)t.y; }

// d * log2(d) for integral d >= 1 held in a float (MUFU lg2).
__device__ __forceinline__ float dlog2d(float d) { return d * __log2f(d); }

// Two floats rounded to BF16 (nearest, ties to even), lo in the low half.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Credit R_u(x) of middle node u to its end x (an L2 reduction, no return).
__device__ __forceinline__ void credit_end(double *Tacc, int x, double r) { atomicAdd(Tacc + x, r); }

constexpr double LN2 = 0.69314718055994530942;

}  // namespace ef

namespace ef {

// ---------------------------------------------------- learned ranking path
// The regression network 16-64-64-1 (ReLU) on standardised node features.
// Parameters in flattened order: W1 [16][64] row-major, b1[64], W2 [64][64]
// row-major (W2[i][j] joins unit i of layer 1 to unit j of layer 2), b2[64],
// w3[64], b3.
constexpr int MLP_F = 16, MLP_H = 64;
constexpr int P_W1 = 0, P_B1 = 1024, P_W2 = 1088, P_B2 = 5184, P_W3 = 5248, P_B3 = 5312, P_N = 5313;

// A model on the device (one allocation): FP32 master parameters, the
// standardisation, Adam moments, the gradient buffer and BF16 copies of the
// weights laid out for the tensor-core fragments (w1t[j][f] = W1[f][j],
// w2t[j][i] = W2[i][j], w2r = W2 row-major).
struct ModelDev {
    float p[P_N];
    float mean[MLP_F], stdv[MLP_F];
    float m[P_N], v[P_N], grad[P_N];
    float loss_sum;
    int32_t step;
    int32_t feature_mode;   // 0: features without triangles, 1: with
    int32_t pad;
    __align__(16) uint16_t w1t[MLP_H * MLP_F];
    __align__(16) uint16_t w2t[MLP_H * MLP_H];
    __align__(16) uint16_t w2r[MLP_H * MLP_H];
};

// Working buffers of the learned path (carved from one allocation).
struct RankScratch {
    float *x;            // n x 16 features
    float *score;        // n predictions
    int32_t *nbr_min, *nbr_max;   // n
    uint64_t *key;       // n selection keys
    int32_t *flag, *pos; // n and n+1: compaction flags and their scan
    int32_t *list;       // n: selected node ids
    int32_t *listL;      // n: candidates and audit nodes
    int32_t *lista;      // n: audit nodes
    int32_t *role;       // n: bit 1 candidate, bit 2 audit
    int32_t *hist;       // 65536 digit counts
    uint64_t *sel;       // selection state: prefix, need, k
    int32_t *scan_tmp;
    double *exact;       // n: exact EF of listL by position
    double *exact_node;  // n: exact EF by node (listed nodes only)
    float *a_score;      // n: audit predictions
    double *a_exact;     // n: audit exact EF
};

}  // namespace ef

// ------------------------------------------------------------ launchers
namespace ef {
// goff, G: a batch's G + 1 graph node offsets on the device (the row pass
// then also checks that no entry leaves its row's graph), else nullptr.
int launch_prep_a(const int32_t *rp, const int32_t *ci, int32_t n, int64_t m, const Scratch &s, const Tune &t,
                  cudaStream_t st, const int64_t *goff = nullptr, int32_t G = 0);
// The out-lists in degree-bin order (bins) or node order.
// With tables, also the hash tables of the out-lists longer than SHORT_MAX
// (cleared here, filled as the lists are written).
int launch_orient(const int32_t *rp, const int32_t *ci, int32_t n, int64_t m, const Scratch &s, const Tune &t,
                  cudaStream_t st, int32_t *nmin = nullptr, int32_t *nmax = nullptr, bool bins = true,
                  bool tables = true);
int launch_big_items(const Scratch &s, int32_t n, cudaStream_t st);
int prepare_kernels();
int prepare_final_tables();   // ln table of the finalize (ef_final.cu), once per device
int64_t device_l2_bytes();   // of the current device (after prepare_kernels ran on it)

// Whether the one-thread row passes may take their rows in work-bin order
// (RowOrder): only when the column array fits in half of L2, so that rows
// visited out of id order cost no extra DRAM traffic.  (BA n = 1M, 44 MB of
// CSR: step 1.10 -> 0.82 ms in bin order; BA n = 16M, 580 MB: 9.9 -> 11.3 ms.)
inline bool rows_in_bins_allowed(int64_t m) { return 4 * m <= device_l2_bytes() / 2; }
int launch_scan(const int32_t *in, int32_t *out, int32_t n, int32_t *tmp, cudaStream_t st);
int launch_ftab(float2 *ftab, int64_t *tq, int32_t *cnt, int64_t cap, cudaStream_t st);
// Device-side check after the row passes: the validation bits (error word,
// symmetry sum, maximum degree above EF_MAX_DEGREE) into cnt[CNT_GATE], and
// OR-ed into *sticky when it is not null.
int launch_gate(int32_t *cnt, int32_t *sticky, cudaStream_t st);
int launch_wedge_small(const int32_t *rp, const int32_t *ci, const Scratch &s, int precision, int32_t n,
                       const Tune &t, cudaStream_t st);
int launch_wedge_big(const int32_t *rp, const int32_t *ci, const Scratch &s, int precision, int wedge_mode,
                     int32_t n, int64_t m, const Tune &t, cudaStream_t st);
int launch_tri_pairs(const Scratch &s, int32_t n, int64_t m, const Tune &t, cudaStream_t st,
                     const int32_t *owner_range = nullptr);
int launch_finalize(const Scratch &s, int precision, int32_t n, const ef_outputs &out, const Tune &t,
                    cudaStream_t st);
// learned path (ef_mlp.cu, ef_rank.cu)
int launch_mlp_infer(const ModelDev *M, const float *x, int32_t n, float *out, int num_sms, cudaStream_t st);
// The same network on rows already standardised and rounded to BF16 (8
// words of two features per row, as launch_features writes them with a
// model): the same predictions, half the bytes read.
int launch_mlp_infer_bf16(const ModelDev *M, const uint32_t *xb, int32_t n, float *out, int num_sms,
                          cudaStream_t st);
int launch_mlp_step(ModelDev *M, const float *x, const float *y, int32_t n, int32_t batch, uint64_t seed, bool sample,
                    bool count_step, bool adam, float lr, uint16_t *acts, int num_sms, cudaStream_t st);
size_t mlp_act_bytes(int32_t batch);
int launch_model_pack(ModelDev *M, cudaStream_t st);
int launch_feature_stats(const float *x, int32_t n, ModelDev *M, double *tmp, cudaStream_t st);
int launch_omega_mm(const int32_t *rp, const int32_t *ci, int32_t n, int64_t m, const Scratch &s,
                    const RankScratch &r, const Tune &t, cudaStream_t st);
// std_model: write the rows standardised with that model's statistics and
// rounded to BF16 into r.x (8 words per row) instead of FP32 features.
int launch_features(const Scratch &s, const RankScratch &r, int32_t n, int mode, const Tune &t, cudaStream_t st,
                    const ModelDev *std_model = nullptr);
int launch_select_top(const RankScratch &r, int32_t n, int64_t k, int bits, const Tune &t, cudaStream_t st);
int launch_bin_nodes(const int32_t *list, int32_t k, const int32_t *kptr, const int32_t *rp, const int32_t *ci,
                     const Scratch &s, int32_t *mark, int32_t n, const Tune &t, cudaStream_t st);
int launch_bin_marked(const int32_t *mark, const Scratch &s, int32_t n, const Tune &t, cudaStream_t st);
// SIR simulation (ef_sir.cu): a batch of at most SIR_BATCH simulations,
// node-major bit words (WB = ceil(B / 32) per node), frontier lists of nodes.
constexpr int SIR_BATCH = 1024;
struct SirState {
    int32_t B, WB;        // simulations of the batch, words per node
    uint32_t *susc;       // n*WB   susceptible (bit s % 32 of word s / 32)
    uint32_t *inf[2];     // n*WB   infected at the start of this step / of the next
    uint32_t *newinf;     // n*WB   infected during this step
    int32_t *cand;        // n*B    smallest successful infector of the step (x * B + s)
    int32_t *parent;      // B*n    infection tree (s * n + v): -1 never infected, the index case itself
    int32_t *front[2];    // n      nodes infected in some simulation, this step / the next
    int32_t *touched;     // n      nodes with a successful try this step
    int32_t *heavy;       // n      frontier nodes of high degree this step
    int32_t *fmark, *tmark;   // n  step stamps deduplicating the appends to front and touched
    int32_t *counts;      // 4      lengths of front[0], front[1], touched, heavy
    int32_t *count, *peak, *peak_step, *length, *fsize;   // B
    uint8_t *done;        // B      1: no infected node left (or never started)
    int32_t *err;         // error bits (ERRB_SIR_ARG)
};
struct SirStep {
    uint64_t seed;        // Philox key
    int64_t sim_base;     // counter word 0 = sim_base + simulation index
    uint64_t beta_thr;    // floor(beta 2^32): a try succeeds when its draw is below
    uint64_t gamma_thr;   // floor(gamma 2^32): recovery
};
int launch_sir_init(const int32_t *index_cases, int32_t n, const uint8_t *immune, int32_t num_sets,
                    const int32_t *imm_set, const SirState &st, const Tune &t, cudaStream_t s);
int launch_sir_step(const int32_t *rp, const int32_t *ci, int32_t n, int32_t step, const SirStep &p,
                    const SirState &st, int64_t *active, const Tune &t, cudaStream_t s);
int launch_sir_close(int32_t steps, const SirState &st, uint8_t *truncated, const Tune &t, cudaStream_t s);
int launch_sir_tree(int32_t n, int32_t depth, int32_t min_size, const SirState &st, int64_t *exact,
                    int64_t *infected, const Tune &t, cudaStream_t s);
int launch_sir_cumulate(int32_t n, int32_t depth, int64_t *spread, const Tune &t, cudaStream_t s);
// shards (ef_shard.cu; the partials' finalize in ef_final.cu)
int launch_shard_range(const int32_t *rp, int32_t n, int64_t m, int32_t shard, int32_t nshards, int32_t *range,
                       cudaStream_t st);
int launch_mark_range(const int32_t *range, int32_t n, int32_t *mark, const Tune &t, cudaStream_t st);
int launch_shard_out(const int32_t *range, const Scratch &s, int precision, int32_t n, const ef_partials &out,
                     const Tune &t, cudaStream_t st);
int launch_finalize_sums(const ef_partials &p, int precision, int32_t n, int32_t frac_bits, const ef_outputs &out,
                         const Tune &t, cudaStream_t st);
int launch_nodes_exact(const int32_t *rp, const int32_t *ci, const Scratch &s, const int32_t *list, int32_t k,
                       const int32_t *kptr, int32_t n, int precision, bool global_tri, const ef_outputs &out,
                       const Tune &t, cudaStream_t st);
int launch_keys_score(const float *score, int32_t n, uint64_t *key, cudaStream_t st);
int launch_roles(const int32_t *cand, int32_t kc, int32_t n, uint64_t seed, uint64_t threshold, int32_t *role,
                 cudaStream_t st);
int launch_compact_role(const int32_t *role, int32_t n, int mask, int32_t *flag, int32_t *pos, int32_t *tmp,
                        int32_t *list, cudaStream_t st);
int launch_exact_keys(const int32_t *L, const int32_t *kL, int32_t kmax, const double *exact, const int32_t *role,
                      double *exact_node, uint64_t *key, cudaStream_t st);
int launch_gather_top(const int32_t *list, int32_t k, const double *exact_node, int32_t *out_idx, double *out_ef,
                      cudaStream_t st);
int launch_gather_audit(const int32_t *list, const int32_t *ka, int32_t kmax, const float *score,
                        const double *exact_node, float *a_score, double *a_exact, cudaStream_t st);
}  // namespace ef
