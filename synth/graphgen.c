/*
 * Seeded synthetic graph generators (host C).
 *
 * Every generator returns an undirected simple graph as a symmetric CSR with
 * int32 indices, sorted rows, no self-loops and no duplicate entries
 * (nnz = 2|E|).  The generators hold no Expected-Force arithmetic: they only
 * build inputs shaped like the paper's workloads (Section 5.1, Table 1): an
 * Erdos-Renyi graph, Barabasi-Albert graphs, a power-law configuration model,
 * Watts-Strogatz graphs (single and as a disjoint-union batch) and R-MAT.
 *
 * Randomness: xoshiro256** (Blackman & Vigna, 2018) seeded through splitmix64
 * (Steele, Lea & Flood, 2014).  Identical seeds give identical graphs on any
 * little- or big-endian 64-bit host; nothing depends on the sign of `char`.
 *
 * Memory ownership: gg_* functions allocate the CSR arrays with malloc and
 * hand them to the caller, who releases them with gg_free.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ RNG */
typedef struct { uint64_t s[4]; } gg_rng;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static void rng_seed(gg_rng *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}
static inline uint64_t rng_next(gg_rng *r) {
    uint64_t *s = r->s;
    uint64_t res = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return res;
}
/* uniform double in [0, 1) with 53 random bits */
static inline double rng_unif(gg_rng *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }
/* uniform integer in [0, k), k >= 1, by rejection of the biased tail */
static inline uint64_t rng_below(gg_rng *r, uint64_t k) {
    uint64_t lim = UINT64_MAX - (UINT64_MAX % k);
    uint64_t x;
    do { x = rng_next(r); } while (x >= lim);
    return x % k;
}

/* ---------------------------------------------------------- edge buffer */
typedef struct { int32_t *u, *v; int64_t len, cap; } gg_edges;

static int edges_push(gg_edges *e, int32_t a, int32_t b) {
    if (e->len == e->cap) {
        int64_t nc = e->cap ? e->cap * 2 : 1024;
        int32_t *nu = (int32_t *)realloc(e->u, (size_t)nc * sizeof(int32_t));
        if (!nu) return -1;
        e->u = nu;
        int32_t *nv = (int32_t *)realloc(e->v, (size_t)nc * sizeof(int32_t));
        if (!nv) return -1;
        e->v = nv;
        e->cap = nc;
    }
    e->u[e->len] = a; e->v[e->len] = b; e->len++;
    return 0;
}
static void edges_free(gg_edges *e) { free(e->u); free(e->v); memset(e, 0, sizeof(*e)); }

/* -------------------------------------------------------- CSR assembly */
static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}
static void sort_row(int32_t *p, int64_t len) {
    if (len < 24) {               /* insertion sort for short rows */
        for (int64_t i = 1; i < len; ++i) {
            int32_t x = p[i]; int64_t j = i - 1;
            while (j >= 0 && p[j] > x) { p[j + 1] = p[j]; --j; }
            p[j + 1] = x;
        }
    } else {
        qsort(p, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

/*
 * Build a symmetric simple CSR from an undirected edge list: both directions
 * are stored, self-loops are dropped, duplicate entries are merged and every
 * row is sorted ascending.  Returns 0 on success, -1 on allocation failure,
 * -2 if the result would not fit in int32 indices.
 */
static int build_csr(int32_t n, const gg_edges *e, int32_t **row_ptr_out, int32_t **col_out, int64_t *nnz_out) {
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t i = 0; i < e->len; ++i) {
        int32_t a = e->u[i], b = e->v[i];
        if (a == b) continue;
        cnt[a + 1]++; cnt[b + 1]++;
    }
    for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    int64_t tot = cnt[n];
    int32_t *col = (int32_t *)malloc((size_t)(tot ? tot : 1) * sizeof(int32_t));
    int64_t *pos = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!col || !pos) { free(cnt); free(col); free(pos); return -1; }
    memcpy(pos, cnt, ((size_t)n + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < e->len; ++i) {
        int32_t a = e->u[i], b = e->v[i];
        if (a == b) continue;
        col[pos[a]++] = b; col[pos[b]++] = a;
    }
    free(pos);
    /* sort + dedupe each row in place, compacting */
    int64_t w = 0;
    int32_t *rp = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!rp) { free(cnt); free(col); return -1; }
    rp[0] = 0;
    for (int32_t r = 0; r < n; ++r) {
        int64_t s = cnt[r], t = cnt[r + 1];
        sort_row(col + s, t - s);
        int64_t row_start = w;
        for (int64_t i = s; i < t; ++i) {
            if (w > row_start && col[w - 1] == col[i]) continue;
            col[w++] = col[i];
        }
        if (w > INT32_MAX) { free(cnt); free(col); free(rp); return -2; }
        rp[r + 1] = (int32_t)w;
    }
    free(cnt);
    *row_ptr_out = rp;
    *col_out = col;
    *nnz_out = w;
    return 0;
}

/* ------------------------------------------------------------ generators */

/* Erdos-Renyi G(n, p) by geometric skipping over the pairs w < v
 * (Batagelj & Brandes 2005, "Efficient generation of large random networks"). */
int gg_erdos_renyi(int32_t n, double p, uint64_t seed, int32_t **row_ptr, int32_t **col, int64_t *nnz) {
    gg_edges e = {0};
    gg_rng r; rng_seed(&r, seed);
    if (p > 0.0 && n > 1) {
        if (p >= 1.0) {
            for (int32_t v = 1; v < n; ++v)
                for (int32_t w = 0; w < v; ++w)
                    if (edges_push(&e, v, w)) { edges_free(&e); return -1; }
        } else {
            double lq = log(1.0 - p);
            int64_t v = 1, w = -1;
            while (v < n) {
                double u = rng_unif(&r);
                w += 1 + (int64_t)floor(log(1.0 - u) / lq);
                while (w >= v && v < n) { w -= v; ++v; }
                if (v < n && edges_push(&e, (int32_t)v, (int32_t)w)) { edges_free(&e); return -1; }
            }
        }
    }
    int rc = build_csr(n, &e, row_ptr, col, nnz);
    edges_free(&e);
    return rc;
}

/* Barabasi-Albert preferential attachment.  The seed graph is the star on
 * nodes 0..m (centre 0); every later node joins with m distinct neighbours
 * drawn with probability proportional to degree, by uniform picks from the
 * list of all edge endpoints so far (Batagelj & Brandes 2005).  Picks that
 * repeat a neighbour already chosen for the same node are redrawn. */
int gg_barabasi_albert(int32_t n, int32_t m, uint64_t seed, int32_t **row_ptr, int32_t **col, int64_t *nnz) {
    if (m < 1 || n < m + 1) return -3;
    gg_rng r; rng_seed(&r, seed);
    int64_t ne = (int64_t)m + (int64_t)(n - m - 1) * m;
    int32_t *ends = (int32_t *)malloc((size_t)(2 * ne) * sizeof(int32_t));
    gg_edges e = {0};
    if (!ends) return -1;
    e.cap = ne; e.u = (int32_t *)malloc((size_t)ne * sizeof(int32_t)); e.v = (int32_t *)malloc((size_t)ne * sizeof(int32_t));
    if (!e.u || !e.v) { free(ends); edges_free(&e); return -1; }
    int64_t ln = 0;
    for (int32_t i = 1; i <= m; ++i) {
        e.u[e.len] = 0; e.v[e.len] = i; e.len++;
        ends[ln++] = 0; ends[ln++] = i;
    }
    int32_t *pick = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    if (!pick) { free(ends); edges_free(&e); return -1; }
    for (int32_t v = m + 1; v < n; ++v) {
        int64_t lim = ln;   /* draw only among endpoints present before v */
        for (int32_t k = 0; k < m; ++k) {
            int32_t t;
            int dup;
            do {
                t = ends[rng_below(&r, (uint64_t)lim)];
                dup = 0;
                for (int32_t q = 0; q < k; ++q) if (pick[q] == t) { dup = 1; break; }
            } while (dup);
            pick[k] = t;
        }
        for (int32_t k = 0; k < m; ++k) {
            e.u[e.len] = v; e.v[e.len] = pick[k]; e.len++;
            ends[ln++] = v; ends[ln++] = pick[k];
        }
    }
    free(pick); free(ends);
    int rc = build_csr(n, &e, row_ptr, col, nnz);
    edges_free(&e);
    return rc;
}

/* Configuration model with a discrete power-law degree sequence
 * P(d) proportional to d^-gamma on [dmin, dmax].  Stubs are matched by a
 * uniform random permutation (Fisher-Yates); self-loops are dropped and
 * multi-edges merged, so realised degrees can fall below the drawn ones.
 * If the drawn degree sum is odd, node n-1 receives one extra stub. */
int gg_powerlaw_cm(int32_t n, double gamma, int32_t dmin, int32_t dmax, uint64_t seed,
                   int32_t **row_ptr, int32_t **col, int64_t *nnz) {
    if (n < 1 || dmin < 1 || dmax < dmin) return -3;
    gg_rng r; rng_seed(&r, seed);
    int32_t nk = dmax - dmin + 1;
    double *cdf = (double *)malloc((size_t)nk * sizeof(double));
    if (!cdf) return -1;
    double acc = 0.0;
    for (int32_t i = 0; i < nk; ++i) { acc += pow((double)(dmin + i), -gamma); cdf[i] = acc; }
    int32_t *deg = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!deg) { free(cdf); return -1; }
    int64_t stubs = 0;
    for (int32_t v = 0; v < n; ++v) {
        double u = rng_unif(&r) * acc;
        int32_t lo = 0, hi = nk - 1;           /* first i with cdf[i] > u */
        while (lo < hi) { int32_t mid = lo + (hi - lo) / 2; if (cdf[mid] > u) hi = mid; else lo = mid + 1; }
        deg[v] = dmin + lo;
        stubs += deg[v];
    }
    free(cdf);
    if (stubs & 1) { deg[n - 1]++; stubs++; }
    int32_t *st = (int32_t *)malloc((size_t)stubs * sizeof(int32_t));
    if (!st) { free(deg); return -1; }
    int64_t k = 0;
    for (int32_t v = 0; v < n; ++v) for (int32_t i = 0; i < deg[v]; ++i) st[k++] = v;
    free(deg);
    for (int64_t i = stubs - 1; i > 0; --i) {
        int64_t j = (int64_t)rng_below(&r, (uint64_t)i + 1);
        int32_t t = st[i]; st[i] = st[j]; st[j] = t;
    }
    gg_edges e = {0};
    e.len = stubs / 2; e.cap = e.len;
    e.u = (int32_t *)malloc((size_t)(e.len ? e.len : 1) * sizeof(int32_t));
    e.v = (int32_t *)malloc((size_t)(e.len ? e.len : 1) * sizeof(int32_t));
    if (!e.u || !e.v) { free(st); edges_free(&e); return -1; }
    for (int64_t i = 0; i < e.len; ++i) { e.u[i] = st[2 * i]; e.v[i] = st[2 * i + 1]; }
    free(st);
    int rc = build_csr(n, &e, row_ptr, col, nnz);
    edges_free(&e);
    return rc;
}

/* Watts-Strogatz edges for one graph (ring lattice with k/2 neighbours per
 * side, each lattice edge (i, i+j) rewired with probability p to (i, w) with
 * w uniform and w != i), appended with an index offset. */
static int ws_edges(gg_edges *e, gg_rng *r, int32_t off, int32_t n, int32_t k, double p) {
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t j = 1; j <= k / 2; ++j) {
            int32_t t = (i + j) % n;
            if (rng_unif(r) < p) {
                int32_t w;
                do { w = (int32_t)rng_below(r, (uint64_t)n); } while (w == i);
                t = w;
            }
            if (edges_push(e, off + i, off + t)) return -1;
        }
    }
    return 0;
}

int gg_watts_strogatz(int32_t n, int32_t k, double p, uint64_t seed, int32_t **row_ptr, int32_t **col, int64_t *nnz) {
    if (n < 3 || k < 2 || k >= n) return -3;
    gg_rng r; rng_seed(&r, seed);
    gg_edges e = {0};
    if (ws_edges(&e, &r, 0, n, k, p)) { edges_free(&e); return -1; }
    int rc = build_csr(n, &e, row_ptr, col, nnz);
    edges_free(&e);
    return rc;
}

/* A batch of G Watts-Strogatz graphs as one disjoint-union CSR.  Graph g has
 * n_g uniform in [nlo, nhi], k_g uniform among the even values in [klo, khi]
 * and rewiring probability p.  graph_off[g] is the first node of graph g and
 * graph_off[G] the total node count (caller passes an array of G+1 int64). */
int gg_ws_batch(int32_t G, int32_t nlo, int32_t nhi, int32_t klo, int32_t khi, double p, uint64_t seed,
                int64_t *graph_off, int32_t **row_ptr, int32_t **col, int64_t *nnz) {
    if (G < 1 || nlo < 3 || nhi < nlo || klo < 2 || khi < klo || khi >= nlo) return -3;
    gg_rng r; rng_seed(&r, seed);
    int32_t nkv = (khi / 2) - ((klo + 1) / 2) + 1;
    int64_t off = 0;
    gg_edges e = {0};
    for (int32_t g = 0; g < G; ++g) {
        int32_t n = nlo + (int32_t)rng_below(&r, (uint64_t)(nhi - nlo + 1));
        int32_t k = 2 * (((klo + 1) / 2) + (int32_t)rng_below(&r, (uint64_t)nkv));
        graph_off[g] = off;
        if (off + n > INT32_MAX) { edges_free(&e); return -2; }
        if (ws_edges(&e, &r, (int32_t)off, n, k, p)) { edges_free(&e); return -1; }
        off += n;
    }
    graph_off[G] = off;
    int rc = build_csr((int32_t)off, &e, row_ptr, col, nnz);
    edges_free(&e);
    return rc;
}

/* R-MAT (Chakrabarti, Zhan & Faloutsos 2004) on 2^scale nodes with
 * edge_factor * 2^scale drawn edges and quadrant probabilities a, b, c
 * (d = 1 - a - b - c).  Self-loops and duplicates are removed. */
int gg_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c, uint64_t seed,
            int32_t **row_ptr, int32_t **col, int64_t *nnz) {
    if (scale < 1 || scale > 30 || edge_factor < 1) return -3;
    gg_rng r; rng_seed(&r, seed);
    int32_t n = (int32_t)1 << scale;
    int64_t ne = (int64_t)edge_factor * n;
    gg_edges e = {0};
    e.cap = ne; e.u = (int32_t *)malloc((size_t)ne * sizeof(int32_t)); e.v = (int32_t *)malloc((size_t)ne * sizeof(int32_t));
    if (!e.u || !e.v) { edges_free(&e); return -1; }
    double ab = a + b, abc = a + b + c;
    for (int64_t i = 0; i < ne; ++i) {
        int32_t u = 0, v = 0;
        for (int32_t l = 0; l < scale; ++l) {
            double x = rng_unif(&r);
            int32_t bu = 0, bv = 0;
            if (x < a) { }
            else if (x < ab) { bv = 1; }
            else if (x < abc) { bu = 1; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu; v = (v << 1) | bv;
        }
        e.u[e.len] = u; e.v[e.len] = v; e.len++;
    }
    int rc = build_csr(n, &e, row_ptr, col, nnz);
    edges_free(&e);
    return rc;
}

/* Build a CSR from caller-provided undirected edges (same cleaning rules). */
int gg_from_edges(int32_t n, int64_t ne, const int32_t *u, const int32_t *v,
                  int32_t **row_ptr, int32_t **col, int64_t *nnz) {
    gg_edges e = {0};
    e.u = (int32_t *)u; e.v = (int32_t *)v; e.len = ne; e.cap = ne;
    for (int64_t i = 0; i < ne; ++i) if (u[i] < 0 || u[i] >= n || v[i] < 0 || v[i] >= n) return -3;
    return build_csr(n, &e, row_ptr, col, nnz);
}

void gg_free(void *p) { free(p); }
