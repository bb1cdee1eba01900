/*
 * Seeded synthetic graph generators (input recipe only).
 *
 * This module draws the synthetic graphs that stand in for the paper's
 * datasets: stochastic block models (SBM), R-MAT graphs and Barabasi-Albert
 * graphs.  It holds none of the embedding method's arithmetic; both the
 * CUDA path and the CPU oracle receive its output (an int32 CSR matrix) as
 * plain input.
 *
 * Every generator returns an undirected, simple graph as a symmetric CSR
 * matrix whose rows are sorted ascending, with no self loops and no
 * duplicate entries (each undirected edge {u,v} appears as (u,v) and (v,u)).
 *
 * Randomness: splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), seeded by the caller.
 *
 * Algorithms:
 *  - SBM: for every block pair, candidate pairs are enumerated in
 *    lexicographic order and skipped geometrically (Batagelj & Brandes,
 *    "Efficient generation of large random networks", Phys. Rev. E 2005).
 *  - R-MAT: each edge descends `scale` levels of the adjacency quadtree with
 *    probabilities (a,b,c,d) (Chakrabarti, Zhan, Faloutsos, SDM 2004);
 *    self loops are dropped, duplicates removed after symmetrising.
 *  - Barabasi-Albert: linear-time preferential attachment through an array
 *    of edge endpoints (Batagelj & Brandes 2005), starting from a complete
 *    graph on m+1 vertices; targets of one new vertex are distinct.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct { uint64_t s; } gg_rng;

static uint64_t gg_next(gg_rng* r) {
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
/* uniform double in [0,1) with 53 random bits */
static double gg_unif(gg_rng* r) { return (double)(gg_next(r) >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, bound) (bound > 0), multiply-shift */
static uint64_t gg_below(gg_rng* r, uint64_t bound) {
    /* 128-bit product via two 64x32 halves keeps this portable C */
    uint64_t x = gg_next(r);
    uint64_t xl = x & 0xffffffffull, xh = x >> 32;
    uint64_t bl = bound & 0xffffffffull, bh = bound >> 32;
    uint64_t ll = xl * bl, lh = xl * bh, hl = xh * bl, hh = xh * bh;
    uint64_t mid = (ll >> 32) + (lh & 0xffffffffull) + (hl & 0xffffffffull);
    return hh + (lh >> 32) + (hl >> 32) + (mid >> 32);
}

/* ---- growable edge list of packed (u << 32 | v) with u < v ---- */
typedef struct { uint64_t* e; int64_t len, cap; } gg_list;

static int gg_push(gg_list* l, uint32_t u, uint32_t v) {
    if (u == v) return 0;
    if (u > v) { uint32_t t = u; u = v; v = t; }
    if (l->len == l->cap) {
        int64_t nc = l->cap ? l->cap * 2 : 1024;
        uint64_t* ne = (uint64_t*)realloc(l->e, (size_t)nc * sizeof(uint64_t));
        if (!ne) return -1;
        l->e = ne; l->cap = nc;
    }
    l->e[l->len++] = ((uint64_t)u << 32) | v;
    return 0;
}

/* LSD radix sort of 64-bit keys, 16 bits per pass */
static int gg_radix_sort(uint64_t* a, int64_t len) {
    uint64_t* tmp = (uint64_t*)malloc((size_t)(len > 0 ? len : 1) * sizeof(uint64_t));
    if (!tmp) return -1;
    int64_t* cnt = (int64_t*)malloc(65536 * sizeof(int64_t));
    if (!cnt) { free(tmp); return -1; }
    uint64_t* src = a; uint64_t* dst = tmp;
    for (int pass = 0; pass < 4; ++pass) {
        int sh = pass * 16;
        memset(cnt, 0, 65536 * sizeof(int64_t));
        for (int64_t i = 0; i < len; ++i) cnt[(src[i] >> sh) & 0xffff]++;
        int64_t s = 0;
        for (int b = 0; b < 65536; ++b) { int64_t c = cnt[b]; cnt[b] = s; s += c; }
        for (int64_t i = 0; i < len; ++i) dst[cnt[(src[i] >> sh) & 0xffff]++] = src[i];
        uint64_t* t = src; src = dst; dst = t;
    }
    /* four passes: result is back in a */
    free(cnt); free(tmp);
    return 0;
}

/* Sort, deduplicate and symmetrise an edge list into CSR.
 * On success *row_ptr (n+1) and *col_idx (nnz) are malloc'ed for the caller. */
static int gg_to_csr(gg_list* l, int32_t n, int32_t** row_ptr, int32_t** col_idx, int64_t* nnz_out) {
    if (gg_radix_sort(l->e, l->len)) return -1;
    int64_t m = 0;
    for (int64_t i = 0; i < l->len; ++i)
        if (i == 0 || l->e[i] != l->e[i - 1]) l->e[m++] = l->e[i];
    int64_t nnz = 2 * m;
    if (nnz > INT32_MAX) return -2;
    int32_t* rp = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t* ci = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    int32_t* fill = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!rp || !ci || !fill) { free(rp); free(ci); free(fill); return -1; }
    for (int64_t k = 0; k < m; ++k) {
        uint32_t u = (uint32_t)(l->e[k] >> 32), v = (uint32_t)l->e[k];
        rp[u + 1]++; rp[v + 1]++;
    }
    for (int32_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
    memcpy(fill, rp, (size_t)n * sizeof(int32_t));
    /* edges are sorted by (u,v): row u receives v ascending; row v receives u
     * ascending too (for fixed v, the u's arrive in increasing order).  Rows
     * mix both sources, so sort each row afterwards. */
    for (int64_t k = 0; k < m; ++k) {
        uint32_t u = (uint32_t)(l->e[k] >> 32), v = (uint32_t)l->e[k];
        ci[fill[u]++] = (int32_t)v;
        ci[fill[v]++] = (int32_t)u;
    }
    free(fill);
    for (int32_t i = 0; i < n; ++i) {
        int32_t b = rp[i], e = rp[i + 1];
        for (int32_t x = b + 1; x < e; ++x) {       /* insertion sort: rows are two sorted runs */
            int32_t key = ci[x], y = x - 1;
            while (y >= b && ci[y] > key) { ci[y + 1] = ci[y]; --y; }
            ci[y + 1] = key;
        }
    }
    *row_ptr = rp; *col_idx = ci; *nnz_out = nnz;
    return 0;
}

void gg_free(void* p) { free(p); }

/* Stochastic block model: `nb` blocks with sizes `sizes`, edge probability
 * p_in inside a block and p_out between blocks. */
int gg_sbm(int32_t nb, const int32_t* sizes, double p_in, double p_out, uint64_t seed,
           int32_t* n_out, int32_t** row_ptr, int32_t** col_idx, int64_t* nnz) {
    gg_rng r = { seed };
    int64_t n = 0;
    int64_t* start = (int64_t*)malloc((size_t)(nb + 1) * sizeof(int64_t));
    if (!start) return -1;
    for (int b = 0; b < nb; ++b) { start[b] = n; n += sizes[b]; }
    start[nb] = n;
    if (n > INT32_MAX) { free(start); return -2; }
    gg_list l = { 0, 0, 0 };
    for (int a = 0; a < nb; ++a) {
        for (int b = a; b < nb; ++b) {
            double p = (a == b) ? p_in : p_out;
            if (p <= 0.0) continue;
            int64_t na = sizes[a], nbb = sizes[b];
            /* candidate pairs indexed 0..total-1 */
            int64_t total = (a == b) ? na * (na - 1) / 2 : na * nbb;
            double lq = log1p(-p);
            int64_t k = -1;
            for (;;) {
                if (p >= 1.0) k += 1;
                else {
                    double u = gg_unif(&r);
                    k += 1 + (int64_t)floor(log1p(-u) / lq);
                }
                if (k >= total || k < 0) break;
                int64_t u_, v_;
                if (a == b) {
                    /* k -> (row, col) of the strict upper triangle, row-major */
                    int64_t row = (int64_t)floor((2.0 * na - 1.0 - sqrt((2.0 * na - 1.0) * (2.0 * na - 1.0) - 8.0 * (double)k)) / 2.0);
                    if (row < 0) row = 0;
                    while (row > 0 && row * (2 * na - row - 1) / 2 > k) --row;
                    while ((row + 1) * (2 * na - row - 2) / 2 <= k) ++row;
                    int64_t off = k - row * (2 * na - row - 1) / 2;
                    u_ = start[a] + row; v_ = start[a] + row + 1 + off;
                } else {
                    u_ = start[a] + k / nbb; v_ = start[b] + k % nbb;
                }
                if (gg_push(&l, (uint32_t)u_, (uint32_t)v_)) { free(l.e); free(start); return -1; }
            }
        }
    }
    free(start);
    *n_out = (int32_t)n;
    int rc = gg_to_csr(&l, (int32_t)n, row_ptr, col_idx, nnz);
    free(l.e);
    return rc;
}

/* R-MAT with 2^scale vertices and edge_factor * 2^scale edge draws. */
int gg_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c, uint64_t seed,
            int32_t* n_out, int32_t** row_ptr, int32_t** col_idx, int64_t* nnz) {
    if (scale < 1 || scale > 30) return -2;
    gg_rng r = { seed };
    int64_t n = (int64_t)1 << scale;
    int64_t draws = (int64_t)edge_factor * n;
    gg_list l = { 0, 0, 0 };
    double ab = a + b, abc = a + b + c;
    for (int64_t e = 0; e < draws; ++e) {
        uint32_t u = 0, v = 0;
        for (int lev = 0; lev < scale; ++lev) {
            double x = gg_unif(&r);
            uint32_t bu = 0, bv = 0;
            if (x < a) { }
            else if (x < ab) bv = 1;
            else if (x < abc) bu = 1;
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu; v = (v << 1) | bv;
        }
        if (gg_push(&l, u, v)) { free(l.e); return -1; }
    }
    *n_out = (int32_t)n;
    int rc = gg_to_csr(&l, (int32_t)n, row_ptr, col_idx, nnz);
    free(l.e);
    return rc;
}

/* Barabasi-Albert: n vertices, each new vertex attaches to m distinct
 * existing vertices chosen proportionally to degree. */
int gg_barabasi_albert(int32_t n, int32_t m, uint64_t seed,
                       int32_t* n_out, int32_t** row_ptr, int32_t** col_idx, int64_t* nnz) {
    if (m < 1 || n < m + 1) return -2;
    gg_rng r = { seed };
    int64_t m0 = m + 1;
    int64_t seed_edges = m0 * (m0 - 1) / 2;
    int64_t total = seed_edges + (int64_t)(n - m0) * m;
    uint32_t* ends = (uint32_t*)malloc((size_t)(2 * total) * sizeof(uint32_t));
    uint32_t* pick = (uint32_t*)malloc((size_t)m * sizeof(uint32_t));
    gg_list l = { 0, 0, 0 };
    if (!ends || !pick) { free(ends); free(pick); return -1; }
    l.cap = total; l.e = (uint64_t*)malloc((size_t)total * sizeof(uint64_t));
    if (!l.e) { free(ends); free(pick); return -1; }
    int64_t ne = 0;
    for (int64_t u = 0; u < m0; ++u)
        for (int64_t v = u + 1; v < m0; ++v) {
            ends[2 * ne] = (uint32_t)u; ends[2 * ne + 1] = (uint32_t)v; ++ne;
            gg_push(&l, (uint32_t)u, (uint32_t)v);
        }
    for (int64_t v = m0; v < n; ++v) {
        int64_t pool = 2 * ne;                 /* endpoints present before v arrives */
        for (int t = 0; t < m; ++t) {
            uint32_t cand;
            int dup;
            do {
                cand = ends[gg_below(&r, (uint64_t)pool)];
                dup = 0;
                for (int q = 0; q < t; ++q) if (pick[q] == cand) { dup = 1; break; }
            } while (dup);
            pick[t] = cand;
        }
        for (int t = 0; t < m; ++t) {
            ends[2 * ne] = (uint32_t)v; ends[2 * ne + 1] = pick[t]; ++ne;
            gg_push(&l, (uint32_t)v, pick[t]);
        }
    }
    free(ends); free(pick);
    *n_out = n;
    int rc = gg_to_csr(&l, n, row_ptr, col_idx, nnz);
    free(l.e);
    return rc;
}
