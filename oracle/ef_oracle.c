/*
 * TEST INFRASTRUCTURE ONLY: plain, slow CPU oracle for the Expected Force
 * EF_2 of every node of an undirected simple graph, in FP64.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use
 * this file.  It shares no code, header or table with the CUDA library.
 *
 * Definitions followed (paper: "Scaling Expected Force", Sections 3.3 and 4):
 *   - a 2-hop transmission cluster rooted at v is a tree with two edges that
 *     contains v; its out-degree d is the number of edges joining a cluster
 *     node to a node outside the cluster (Section 3.3);
 *   - EF(v) is the entropy of the normalised cluster degrees d_c / sum d_c over
 *     the clusters credited to v (Eq. 1), natural logarithm;
 *   - Algorithm 1 enumerates each cluster once as a triple (i, v, j), i < j
 *     neighbours of the middle node v, takes d = |Adj v|+|Adj i|+|Adj j|-4,
 *     minus 2 more when i and j are adjacent, and credits the degree once to
 *     i, once to j and twice to v.
 *
 * Readings where the paper is silent: a cluster of degree 0 counts in the
 * histogram and contributes 0 to the entropy (0 log 0 = 0); a node whose
 * cluster degrees sum to 0 (or that has no clusters) is degenerate and gets
 * EF = 0 with its flag set to 1.
 *
 * Return codes: 0 ok, -1 allocation failure, -2 invalid argument.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* library primitive: is `x` in the sorted adjacency row of `v`? */
static int adjacent(const int32_t *row_ptr, const int32_t *col_idx, int32_t v, int32_t x) {
    const int32_t *row = col_idx + row_ptr[v];
    size_t len = (size_t)(row_ptr[v + 1] - row_ptr[v]);
    return bsearch(&x, row, len, sizeof(int32_t), cmp_i32) != NULL;
}

/* ------------------------------------------------ per-node histogram H_v */
/* Open-addressing map from a cluster degree d to its count H_v(d). */
typedef struct { int32_t *key; int64_t *cnt; int32_t cap, size; } hist_t;

static int hist_add(hist_t *h, int32_t d, int64_t c) {
    if (2 * (h->size + 1) > h->cap) {
        int32_t nc = h->cap ? 2 * h->cap : 8;
        int32_t *nk = (int32_t *)malloc((size_t)nc * sizeof(int32_t));
        int64_t *nv = (int64_t *)calloc((size_t)nc, sizeof(int64_t));
        if (!nk || !nv) { free(nk); free(nv); return -1; }
        for (int32_t i = 0; i < nc; ++i) nk[i] = -1;
        for (int32_t i = 0; i < h->cap; ++i) {
            if (h->key[i] < 0) continue;
            uint32_t p = ((uint32_t)h->key[i] * 2654435761u) & (uint32_t)(nc - 1);
            while (nk[p] >= 0) p = (p + 1) & (uint32_t)(nc - 1);
            nk[p] = h->key[i]; nv[p] = h->cnt[i];
        }
        free(h->key); free(h->cnt);
        h->key = nk; h->cnt = nv; h->cap = nc;
    }
    uint32_t p = ((uint32_t)d * 2654435761u) & (uint32_t)(h->cap - 1);
    while (h->key[p] >= 0 && h->key[p] != d) p = (p + 1) & (uint32_t)(h->cap - 1);
    if (h->key[p] < 0) { h->key[p] = d; h->size++; }
    h->cnt[p] += c;
    return 0;
}

/* Entropy of one histogram per Eq. 1, taking every credited cluster as one
 * item with normalised degree d / S.  Also returns N = sum H(d),
 * S = sum H(d) d and T = sum H(d) d ln d.  Degrees are visited in ascending
 * order so that the FP64 sums are reproducible. */
static int entropy_of(const int32_t *keys, const int64_t *cnts, int32_t k,
                      int64_t *N, int64_t *S, double *T, double *EF, uint8_t *flag) {
    int64_t n_ = 0, s_ = 0;
    double t_ = 0.0;
    for (int32_t i = 0; i < k; ++i) {
        n_ += cnts[i];
        s_ += cnts[i] * (int64_t)keys[i];
        if (keys[i] > 0) t_ += (double)cnts[i] * ((double)keys[i] * log((double)keys[i]));
    }
    double ef = 0.0;
    uint8_t fl = 0;
    if (s_ == 0) {
        fl = 1;
    } else {
        double Sd = (double)s_;
        for (int32_t i = 0; i < k; ++i) {
            if (keys[i] == 0) continue;             /* 0 log 0 = 0 */
            double pbar = (double)keys[i] / Sd;     /* normalised cluster degree */
            ef -= (double)cnts[i] * pbar * log(pbar);
        }
    }
    if (N) *N = n_;
    if (S) *S = s_;
    if (T) *T = t_;
    if (EF) *EF = ef;
    if (flag) *flag = fl;
    return 0;
}

typedef struct { int32_t k; int64_t c; } kc_t;
static int cmp_kc(const void *a, const void *b) {
    int32_t x = ((const kc_t *)a)->k, y = ((const kc_t *)b)->k;
    return (x > y) - (x < y);
}

static int hist_entropy(const hist_t *h, int64_t *N, int64_t *S, double *T, double *EF, uint8_t *flag) {
    kc_t *kv = (kc_t *)malloc((size_t)(h->size ? h->size : 1) * sizeof(kc_t));
    if (!kv) return -1;
    int32_t k = 0;
    for (int32_t i = 0; i < h->cap; ++i) if (h->key[i] >= 0) { kv[k].k = h->key[i]; kv[k].c = h->cnt[i]; ++k; }
    qsort(kv, (size_t)k, sizeof(kc_t), cmp_kc);
    int32_t *keys = (int32_t *)malloc((size_t)(k ? k : 1) * sizeof(int32_t));
    int64_t *cnts = (int64_t *)malloc((size_t)(k ? k : 1) * sizeof(int64_t));
    if (!keys || !cnts) { free(kv); free(keys); free(cnts); return -1; }
    for (int32_t i = 0; i < k; ++i) { keys[i] = kv[i].k; cnts[i] = kv[i].c; }
    entropy_of(keys, cnts, k, N, S, T, EF, flag);
    free(kv); free(keys); free(cnts);
    return 0;
}

static int check_csr(int32_t n, const int32_t *row_ptr, const int32_t *col_idx) {
    if (n < 0 || !row_ptr || (n > 0 && row_ptr[0] != 0)) return -2;
    for (int32_t v = 0; v < n; ++v) {
        if (row_ptr[v + 1] < row_ptr[v]) return -2;
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            if (col_idx[e] < 0 || col_idx[e] >= n || col_idx[e] == v) return -2;
            if (e > row_ptr[v] && col_idx[e] <= col_idx[e - 1]) return -2;
        }
    }
    return 0;
}

/*
 * Algorithm 1, literally: Phase 1 materialises the set C of all triples
 * (i, v, j); Phase 2 takes each cluster's degree and updates the histograms
 * of its three members; Phase 3 takes the entropy of every histogram.
 * Outputs (each may be NULL): N[v] = number of credited clusters,
 * S[v] = sum of credited degrees, T[v] = sum of d ln d over credits,
 * EF[v], flag[v] (1 = degenerate).
 */
int ef_oracle_alg1(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                   int64_t *N, int64_t *S, double *T, double *EF, uint8_t *flag) {
    if (check_csr(n, row_ptr, col_idx)) return -2;
    /* Phase 1: cluster generation */
    int64_t W = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t D = row_ptr[v + 1] - row_ptr[v];
        W += D * (D - 1) / 2;
    }
    int32_t *C = (int32_t *)malloc((size_t)(W ? W : 1) * 3 * sizeof(int32_t));
    if (!C) return -1;
    int64_t c = 0;
    for (int32_t v = 0; v < n; ++v)
        for (int32_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a)
            for (int32_t b = row_ptr[v]; b < row_ptr[v + 1]; ++b) {
                int32_t i = col_idx[a], j = col_idx[b];
                if (!(i < j)) continue;
                C[3 * c] = i; C[3 * c + 1] = v; C[3 * c + 2] = j; ++c;
            }
    /* Phase 2: cluster degrees and histogram updates */
    hist_t *H = (hist_t *)calloc((size_t)(n ? n : 1), sizeof(hist_t));
    if (!H) { free(C); return -1; }
    int rc = 0;
    for (int64_t q = 0; q < W && !rc; ++q) {
        int32_t i = C[3 * q], v = C[3 * q + 1], j = C[3 * q + 2];
        int32_t d = (row_ptr[v + 1] - row_ptr[v]) + (row_ptr[i + 1] - row_ptr[i]) + (row_ptr[j + 1] - row_ptr[j]) - 4;
        if (adjacent(row_ptr, col_idx, j, i)) d -= 2;
        rc |= hist_add(&H[i], d, 1);
        rc |= hist_add(&H[j], d, 1);
        rc |= hist_add(&H[v], d, 2);
    }
    free(C);
    /* Phase 3: entropy of each histogram */
    for (int32_t v = 0; v < n && !rc; ++v) {
        int64_t nv = 0, sv = 0; double tv = 0, ev = 0; uint8_t fv = 0;
        rc = hist_entropy(&H[v], &nv, &sv, &tv, &ev, &fv);
        if (N) N[v] = nv;
        if (S) S[v] = sv;
        if (T) T[v] = tv;
        if (EF) EF[v] = ev;
        if (flag) flag[v] = fv;
    }
    for (int32_t v = 0; v < n; ++v) { free(H[v].key); free(H[v].cnt); }
    free(H);
    return rc ? -1 : 0;
}

/*
 * The vertex-centric formulation (Section 4, the original per-node method):
 * for a seed s, visit every cluster credited to s and build its histogram.
 * The clusters of s, with the multiplicities Algorithm 1 gives them, are the
 * ordered two-step transmission sequences from s: s infects a neighbour a,
 * then either s infects another neighbour b (trees s-a, s-b; each unordered
 * pair is reached in both orders, hence weight 2 for a middle node) or a
 * infects a neighbour b != s (tree s-a-b, s at an end, weight 1).  Cluster
 * degrees use the degree formula of Algorithm 1 with its triangle test.
 *
 * Per node it also returns t[s], the number of triangles through s (pairs
 * of adjacent neighbours).  Runs the seeds in parallel with OpenMP dynamic
 * scheduling in chunks of 2 (Section 4.1) on `threads` threads (<=0: all).
 */
static int vertex_one(int32_t s, const int32_t *row_ptr, const int32_t *col_idx, int64_t *Hd,
                      int32_t *touched, int64_t *N, int64_t *S, double *T, double *EF, uint8_t *flag,
                      int64_t *tri, int32_t *out_keys, int64_t *out_cnts, int32_t *out_k) {
    int32_t ntouch = 0;
    int32_t Ds = row_ptr[s + 1] - row_ptr[s];
    int64_t tcount = 0;
    for (int32_t ea = row_ptr[s]; ea < row_ptr[s + 1]; ++ea) {
        int32_t a = col_idx[ea];
        int32_t Da = row_ptr[a + 1] - row_ptr[a];
        /* s infects a, then s infects b */
        for (int32_t eb = row_ptr[s]; eb < row_ptr[s + 1]; ++eb) {
            int32_t b = col_idx[eb];
            if (b == a) continue;
            int32_t Db = row_ptr[b + 1] - row_ptr[b];
            int32_t d = Ds + Da + Db - 4;
            if (adjacent(row_ptr, col_idx, a, b)) { d -= 2; if (a < b) ++tcount; }
            if (Hd[d]++ == 0) touched[ntouch++] = d;
        }
        /* s infects a, then a infects b */
        for (int32_t eb = row_ptr[a]; eb < row_ptr[a + 1]; ++eb) {
            int32_t b = col_idx[eb];
            if (b == s) continue;
            int32_t Db = row_ptr[b + 1] - row_ptr[b];
            int32_t d = Ds + Da + Db - 4;
            if (adjacent(row_ptr, col_idx, s, b)) d -= 2;
            if (Hd[d]++ == 0) touched[ntouch++] = d;
        }
    }
    qsort(touched, (size_t)ntouch, sizeof(int32_t), cmp_i32);
    int64_t *cnts = (int64_t *)malloc((size_t)(ntouch ? ntouch : 1) * sizeof(int64_t));
    if (!cnts) return -1;
    for (int32_t i = 0; i < ntouch; ++i) cnts[i] = Hd[touched[i]];
    entropy_of(touched, cnts, ntouch, N, S, T, EF, flag);
    if (out_k) {
        for (int32_t i = 0; i < ntouch; ++i) { out_keys[i] = touched[i]; out_cnts[i] = cnts[i]; }
        *out_k = ntouch;
    }
    for (int32_t i = 0; i < ntouch; ++i) Hd[touched[i]] = 0;
    free(cnts);
    if (tri) *tri = tcount;
    return 0;
}

int ef_oracle_vertex(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                     int64_t k, const int32_t *nodes, int32_t threads,
                     int64_t *N, int64_t *S, double *T, double *EF, uint8_t *flag, int64_t *tri) {
    if (check_csr(n, row_ptr, col_idx)) return -2;
    int32_t maxdeg = 0;
    for (int32_t v = 0; v < n; ++v) if (row_ptr[v + 1] - row_ptr[v] > maxdeg) maxdeg = row_ptr[v + 1] - row_ptr[v];
    for (int64_t q = 0; q < k; ++q) if (nodes[q] < 0 || nodes[q] >= n) return -2;
    size_t range = (size_t)3 * (size_t)maxdeg + 1;
    int rc = 0;
#ifdef _OPENMP
    if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel num_threads(threads) reduction(|:rc)
#endif
    {
        int64_t *Hd = (int64_t *)calloc(range, sizeof(int64_t));
        int32_t *touched = (int32_t *)malloc(range * sizeof(int32_t));
        if (!Hd || !touched) rc |= 1;
        else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 2)
#endif
            for (int64_t q = 0; q < k; ++q) {
                int32_t s = nodes[q];
                rc |= vertex_one(s, row_ptr, col_idx, Hd, touched,
                                 N ? &N[q] : NULL, S ? &S[q] : NULL, T ? &T[q] : NULL,
                                 EF ? &EF[q] : NULL, flag ? &flag[q] : NULL, tri ? &tri[q] : NULL,
                                 NULL, NULL, NULL) ? 1 : 0;
            }
        }
        free(Hd); free(touched);
    }
    return rc ? -1 : 0;
}

/* Histogram H_s of one seed (vertex-centric): writes up to `cap` distinct
 * degrees ascending with their counts; returns the number of distinct
 * degrees, or a negative code. */
int ef_oracle_vertex_hist(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t s,
                          int32_t cap, int32_t *out_d, int64_t *out_c) {
    if (check_csr(n, row_ptr, col_idx) || s < 0 || s >= n) return -2;
    int32_t maxdeg = 0;
    for (int32_t v = 0; v < n; ++v) if (row_ptr[v + 1] - row_ptr[v] > maxdeg) maxdeg = row_ptr[v + 1] - row_ptr[v];
    size_t range = (size_t)3 * (size_t)maxdeg + 1;
    int64_t *Hd = (int64_t *)calloc(range, sizeof(int64_t));
    int32_t *touched = (int32_t *)malloc(range * sizeof(int32_t));
    int32_t *keys = (int32_t *)malloc(range * sizeof(int32_t));
    int64_t *cnts = (int64_t *)malloc(range * sizeof(int64_t));
    int32_t k = 0;
    int rc = -1;
    if (Hd && touched && keys && cnts) {
        rc = vertex_one(s, row_ptr, col_idx, Hd, touched, NULL, NULL, NULL, NULL, NULL, NULL, keys, cnts, &k);
        if (rc == 0) {
            for (int32_t i = 0; i < k && i < cap; ++i) { out_d[i] = keys[i]; out_c[i] = cnts[i]; }
            rc = k;
        }
    }
    free(Hd); free(touched); free(keys); free(cnts);
    return rc;
}

/* Histograms of Algorithm 1 for one node: runs Phases 1-2 literally and
 * returns H_s the same way as ef_oracle_vertex_hist. */
int ef_oracle_alg1_hist(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t s,
                        int32_t cap, int32_t *out_d, int64_t *out_c) {
    if (check_csr(n, row_ptr, col_idx) || s < 0 || s >= n) return -2;
    hist_t h = {0};
    int rc = 0;
    for (int32_t v = 0; v < n && !rc; ++v)
        for (int32_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a)
            for (int32_t b = row_ptr[v]; b < row_ptr[v + 1]; ++b) {
                int32_t i = col_idx[a], j = col_idx[b];
                if (!(i < j)) continue;
                if (i != s && j != s && v != s) continue;
                int32_t d = (row_ptr[v + 1] - row_ptr[v]) + (row_ptr[i + 1] - row_ptr[i]) + (row_ptr[j + 1] - row_ptr[j]) - 4;
                if (adjacent(row_ptr, col_idx, j, i)) d -= 2;
                if (i == s) rc |= hist_add(&h, d, 1);
                if (j == s) rc |= hist_add(&h, d, 1);
                if (v == s) rc |= hist_add(&h, d, 2);
            }
    int32_t k = 0;
    if (!rc) {
        kc_t *kv = (kc_t *)malloc((size_t)(h.size ? h.size : 1) * sizeof(kc_t));
        if (!kv) rc = -1;
        else {
            for (int32_t i = 0; i < h.cap; ++i) if (h.key[i] >= 0) { kv[k].k = h.key[i]; kv[k].c = h.cnt[i]; ++k; }
            qsort(kv, (size_t)k, sizeof(kc_t), cmp_kc);
            for (int32_t i = 0; i < k && i < cap; ++i) { out_d[i] = kv[i].k; out_c[i] = kv[i].c; }
            free(kv);
        }
    }
    free(h.key); free(h.cnt);
    return rc ? -1 : k;
}

/* Plain definition of per-node triangle counts: t[v] = number of pairs of
 * adjacent neighbours of v. */
int ef_oracle_triangles(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int64_t *t) {
    if (check_csr(n, row_ptr, col_idx)) return -2;
    for (int32_t v = 0; v < n; ++v) {
        int64_t c = 0;
        for (int32_t a = row_ptr[v]; a < row_ptr[v + 1]; ++a)
            for (int32_t b = a + 1; b < row_ptr[v + 1]; ++b)
                if (adjacent(row_ptr, col_idx, col_idx[a], col_idx[b])) ++c;
        t[v] = c;
    }
    return 0;
}

int ef_oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
