/*
 * GEMPE CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 restatement of one GEMPE epoch
 * (Boehm & Plant, "Massively Parallel Graph Drawing and Representation
 * Learning", arXiv 2011.03479).  Only the tests, the package's smoke check
 * and the benchmark's CPU-baseline leg load this file; the CUDA engine never
 * calls it, includes it or shares a line of code with it.
 *
 * What each function follows:
 *   orc_h_basic            Eq. 1 (basic entropy of the adjacency matrix)
 *   orc_dl                 Sec. II.B: description lengths dl+ / dl- of the
 *                          sigmoid s+ = 1/2 - 1/2 erf((delta-mu)/(sqrt2 sigma))
 *   orc_parabola           Eq. 4 (w) and Eq. 5 (d) for edges, and the same
 *                          formulas with the marked "-" signs turned into "+"
 *                          for non-edges (Sec. II.C)
 *   orc_epoch              one iteration of Fig. 4: zero y,z; edge parabolas;
 *                          sampled non-edges (Fig. 2 semantics, Sec. III.C;
 *                          Philox draws, or Sec. III.C's LCG with rng 1);
 *                          Eq. 3 numerators/denominators; x_i := y_i / z_i;
 *                          distance histograms (Sec. III.F)
 *   orc_sigma_fit          Sec. III.F: bisection for dPE/dsigma = 0 on the
 *                          edge / non-edge distance histograms, mu fixed
 *   orc_loss_exact         Eq. 2 at a given sigma, all n(n-1)/2 pairs
 *   orc_dpe_dsigma_exact,  Eq. 2 differentiated in sigma over all pairs, and
 *   orc_sigma_fit_exact    its zero (the slope minimising Eq. 2, mu fixed)
 *   orc_loss_sampled       Eq. 2 estimated from all edges plus sampled
 *                          non-edges weighted to the non-edge count
 *   orc_edge_terms_*       the edge part of Eq. 3 in the paper's edge-list
 *                          form (Fig. 4) and in the per-vertex CSR form
 *   orc_surrogate_L        sum of dl over a frozen pair list (for the
 *                          gradient identity of Eq. 3)
 *   orc_vertex_terms       Eq. 3's sums of chosen vertices alone, with the
 *                          samples of orc_epoch (checks at full sizes)
 *   orc_epoch_range        the terms of a range of anchors (Sec. III.E's
 *                          split of Eq. 3's sums over workers)
 *
 * Choices where the paper is silent (the "readings"):
 *   - negative samples are drawn per vertex, k per vertex per epoch, with a
 *     Philox4x32-10 counter stream; a draw g is rejected when g == i or
 *     (i,g) is an edge, and redrawn at most max_retries times (Fig. 2 loops
 *     without bound);
 *   - membership is exact (binary search in the sorted CSR row) instead of
 *     the lossy byte-map hash of Sec. III.C;
 *   - w_formula 0 ("derived"): the first term of Eq. 4 uses 1/(pi ln2), the
 *     factor that matching the second derivative actually gives; w_formula 1
 *     ("printed") keeps the 2/(pi ln2) printed in Eq. 4.  Eq. 5 is used as
 *     printed in both cases;
 *   - clamp_neg_d: d := max(d, 0);
 *   - x_i is left unchanged when z_i < z_min;
 *   - non-edge histogram weight of a sample anchored at i is
 *     (n-1-deg_i) / (2 * accepted_i); edges are binned once (j > i) with
 *     weight 1; bin = min(floor(delta / (hist_max/B)), B-1), value = centre;
 *   - sigma bisection runs in log sigma on [1e-3, 1e3]; without a sign change
 *     the bracket end with the lower entropy is taken.
 *
 * Counter-based random numbers (Philox4x32-10, Salmon, Moraes, Dror & Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC 2011), key =
 * (seed_lo, seed_hi); counter words:
 *   initial positions  (i, q, 0, 0x0A000000)         -> coordinates 4q..4q+3
 *   epoch samples      (i, epoch, t>>2, 0x0B000000|a) -> word t&3 (slot t,
 *                      attempt a: one call serves the attempt a of four slots)
 *   loss samples       (i, epoch, t>>2, 0x0E000000|a) -> word t&3
 *   block partners     (tile, epoch, p>>2, 0x0D000000) -> word p&3
 *   per-slot samples   (e>>2, epoch, 0, 0x0C000000|a)  -> word e&3 (Sec. III.C's
 *                      policy: one sample per CSR slot e, anchored at its row)
 *   slope samples      (i, epoch, t>>2, 0x0F000000|a) -> word t&3 (the separate
 *                      histogram pass of Sec. III.F)
 *   renaming           (period, 0, 0, 0x09000000)     -> words 0, 1 (byte-map
 *                      membership, Sec. III.C)
 *   LCG seeds (rng 1)  (i, epoch, t>>2, 0x08000000)   -> word t&3: the state of
 *                      sample slot t of vertex i; (e>>2, epoch, 0, 0x07000000)
 *                      -> word e&3: the state of CSR slot e (per-slot policy)
 * A 32-bit word r maps to vertex floor(r * n / 2^32); with rng 1 attempt a of
 * a slot draws lcg_vertex of the slot's state advanced a + 1 times.
 *
 * Block sampling (the representation-learning form): vertices are cut into
 * tiles of T consecutive ids; every vertex of a tile takes the same P
 * partners, drawn per tile and epoch.  A pair (i, g) whose partner is i
 * itself or a neighbour of i is masked (skipped, not redrawn); the unmasked
 * partners of i are its sampled non-edges for the epoch, with histogram
 * weight (n-1-deg_i) / (2 * unmasked_i).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* The same source also builds the timed CPU baseline with OpenMP
 * (-fopenmp): the vertex loop and the tile loop of orc_epoch then run over
 * all host threads, every addition into a shared sum becomes an atomic
 * addition, and the per-thread counters are added up at the end.  Built
 * without OpenMP (the parity reference) the pragmas are ignored and the
 * loops run in order, one vertex after another. */
#ifdef _OPENMP
#include <omp.h>
#define ORC_ATOMIC _Pragma("omp atomic")
#else
#define ORC_ATOMIC
#endif

/* Host threads the build runs orc_epoch on (1 without OpenMP). */
int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define ORC_LN2 0.69314718055994530942
#define ORC_PI 3.14159265358979323846
#define ORC_SQRT2 1.41421356237309504880

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                       */
/* ------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = { ctr[0], ctr[1], ctr[2], ctr[3] };
    uint32_t k[2] = { key[0], key[1] };
    for (int r = 0; r < 10; ++r) {
        philox_round(c, k);
        k[0] += 0x9E3779B9u;   /* Weyl sequence increments */
        k[1] += 0xBB67AE85u;
    }
    memcpy(out, c, sizeof c);
}

static uint32_t draw_vertex(uint32_t r, uint32_t n) { return (uint32_t)(((uint64_t)r * n) >> 32); }

/* Sec. III.C's generator for the non-edge partners (rng = 1): a 32-bit
 * linear congruential generator with multiplier 1103515245 and increment 1,
 * state := state * 1103515245 + 1 (mod 2^32), advanced before every draw as
 * Fig. 2 advances its state vector. */
static uint32_t lcg_next(uint32_t s) { return s * 1103515245u + 1u; }

/* Fig. 2's map of a state to a vertex, in FP32 with one rounding per
 * operation: the low 23 bits of the state as the mantissa of a float f in
 * [1, 2), then f * n - n, rounded to the nearest integer (ties to even).
 * Reading: the rounding can reach n, which is taken as vertex 0 (so every
 * vertex gets an interval of width one); for n > 2^23 only 2^23 vertices are
 * reachable, as with the paper's 23-bit mantissa. */
static int32_t lcg_vertex(uint32_t s, int32_t n) {
    uint32_t bits = 0x3F800000u | (s & 0x007FFFFFu);
    float f, nf = (float)n;
    memcpy(&f, &bits, sizeof f);
    float t = f * nf;
    t = t - nf;
    int32_t g = (int32_t)rintf(t);
    if (g >= n) g -= n;
    return g;
}

/* Inspection: the generator's next state and the vertex of a state. */
uint32_t orc_lcg_next(uint32_t s) { return lcg_next(s); }
int32_t orc_lcg_vertex(uint32_t s, int32_t n) { return lcg_vertex(s, n); }

static uint32_t philox_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int word) {
    uint32_t ctr[4] = { c0, c1, c2, c3 };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[word];
}

/* Initial positions (Fig. 4: uniform random), U[-R, R) in FP32. */
void orc_init_positions(int32_t n, int32_t d, uint64_t seed, float range, float* x) {
    for (int32_t i = 0; i < n; ++i)
        for (int32_t c = 0; c < d; ++c) {
            uint32_t r = philox_word(seed, (uint32_t)i, (uint32_t)(c / 4), 0u, 0x0A000000u, c % 4);
            double unit = (double)(r >> 8) * (1.0 / 8388608.0) - 1.0;   /* exact in [-1,1) */
            x[(int64_t)i * d + c] = (float)(unit * (double)range);       /* one rounding */
        }
}

/* ------------------------------------------------------------------ */
/* Graph membership: binary search in the sorted CSR row               */
/* ------------------------------------------------------------------ */
int orc_is_edge(const int32_t* row_ptr, const int32_t* col_idx, int32_t i, int32_t j) {
    int32_t lo = row_ptr[i], hi = row_ptr[i + 1];
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (col_idx[mid] == j) return 1;
        if (col_idx[mid] < j) lo = mid + 1; else hi = mid;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Eq. 1 and Sec. II.B                                                  */
/* ------------------------------------------------------------------ */
double orc_h_basic(double n, double m) {
    double N = 0.5 * n * (n - 1.0);
    double p = m / N, q = (N - m) / N;
    double h = 0.0;
    if (p > 0.0) h -= p * log2(p);
    if (q > 0.0) h -= q * log2(q);
    return h;
}

/* Laplace's continued fraction for the Mills ratio: with
 * Q(u)/phi(u) = 1/(u + 1/(u + 2/(u + 3/(u + ...)))), the tail ratio
 * phi(u)/Q(u) equals u + T(u), T(u) = 1/(u + 2/(u + 3/(u + ...))).
 * Used only for u >= 25 where erfc underflows in double precision. */
static double mills_tail_T(double u) {
    double t = u;
    for (int k = 80; k >= 2; --k) t = u + (double)k / t;
    return 1.0 / t;
}

/* phi(u) / Q(u) with Q the upper normal tail, Q(u) = 1/2 erfc(u/sqrt2). */
static double inv_mills(double u) {
    if (u >= 25.0) return u + mills_tail_T(u);
    double phi = exp(-0.5 * u * u) / sqrt(2.0 * ORC_PI);
    return phi / (0.5 * erfc(u / ORC_SQRT2));
}

/* -log2 Q(u) */
static double neg_log2_Q(double u) {
    if (u >= 25.0) {
        /* Q = phi(u) / (u + T(u)) */
        double lnq = -0.5 * u * u - 0.5 * log(2.0 * ORC_PI) - log(u + mills_tail_T(u));
        return -lnq / ORC_LN2;
    }
    if (u < 0.0)      /* Q(u) = 1 - Q(-u) close to 1: keep the digits of Q(-u) */
        return -log1p(-0.5 * erfc(-u / ORC_SQRT2)) / ORC_LN2;
    return -log2(0.5 * erfc(u / ORC_SQRT2));
}

/* dl+ (is_edge = 1) or dl- (is_edge = 0) of distance delta. */
double orc_dl(double delta, double mu, double sigma, int is_edge) {
    double u = (delta - mu) / sigma;
    /* s+ = 1/2 - 1/2 erf(u/sqrt2) = Q(u);  s- = 1/2 + 1/2 erf(u/sqrt2) = Q(-u) */
    return is_edge ? neg_log2_Q(u) : neg_log2_Q(-u);
}

/* ------------------------------------------------------------------ */
/* Eq. 4 / Eq. 5: the parabola w (delta - d)^2 of one pair              */
/* ------------------------------------------------------------------ */
void orc_parabola(double delta, double mu, double sigma, int is_edge, int w_formula, int clamp_neg_d,
                  double* d_out, double* w_out) {
    const double c1 = (w_formula == 1) ? 2.0 : 1.0;       /* first-term factor of Eq. 4 */
    const double u = (delta - mu) / sigma;
    const double sgn = is_edge ? -1.0 : 1.0;              /* the red operators of Eq. 4/5 */
    double w, d;
    if ((is_edge && u < 25.0) || (!is_edge && u > -25.0)) {
        /* Eq. 4 / 5 as printed, with 1 -/+ erf(x) evaluated as erfc(+/-x) */
        const double e = exp(-(delta - mu) * (delta - mu) / (2.0 * sigma * sigma));
        const double D = is_edge ? erfc(u / ORC_SQRT2) : erfc(-u / ORC_SQRT2);
        const double a = c1 / (ORC_PI * ORC_LN2);
        const double b = 1.0 / (sqrt(2.0 * ORC_PI) * ORC_LN2);
        w = a * e * e / (sigma * sigma * D * D) + sgn * b * (delta - mu) * e / (sigma * sigma * sigma * D);
        d = delta + sgn * b * e / (w * sigma * D);
    } else {
        /* far tail (erfc underflows): same quantities through the Mills
         * ratio, h = phi(v)/Q(v), v = u for edges and -u for non-edges. */
        const double v = is_edge ? u : -u;
        const double h = v + mills_tail_T(v);
        /* in Eq. 4 the first term equals c1 h^2 / (2 ln2 sigma^2) and the
         * second v h / (2 ln2 sigma^2) with the operator sign folded into v */
        w = (c1 * h * h - v * h) / (2.0 * ORC_LN2 * sigma * sigma);
        d = delta + sgn * h / (2.0 * ORC_LN2 * sigma * w);
    }
    if (clamp_neg_d && d < 0.0) d = 0.0;
    *d_out = d;
    *w_out = w;
}

/* ------------------------------------------------------------------ */
/* Eq. 3 contribution of one pair to vertex a (partner b)               */
/* ------------------------------------------------------------------ */
static double dist(const double* x, int32_t d, int64_t a, int64_t b) {
    double s = 0.0;
    for (int32_t c = 0; c < d; ++c) {
        double t = x[a * d + c] - x[b * d + c];
        s += t * t;
    }
    return sqrt(s);
}

/* absd (optional) collects |w (x_b + s (x_a - x_b)) - w x_a| = w |s - 1| delta,
 * the size of the pair's term in y_a - z_a x_a: the scale against which the
 * rounding of a cancelling sum is judged. */
static double* g_absd = NULL;

static void add_wm_term(double* y, double* z, const double* x, int32_t d, int64_t a, int64_t b,
                        double delta, double dd, double w) {
    if (!(w > 0.0)) return;   /* an underflowed weight contributes nothing */
    double s = (delta != 0.0) ? dd / delta : 0.0;
    for (int32_t c = 0; c < d; ++c) {
        double t = w * (x[b * d + c] + s * (x[a * d + c] - x[b * d + c]));
        ORC_ATOMIC y[a * d + c] += t;
    }
    ORC_ATOMIC z[a] += w;
    if (g_absd) {
        double t = w * fabs(s - 1.0) * delta;
        ORC_ATOMIC g_absd[a] += t;
    }
}

static int32_t hist_bin(double delta, int32_t B, double hist_max) {
    double f = floor(delta / (hist_max / (double)B));
    if (f >= (double)(B - 1)) return B - 1;
    if (f < 0.0) return 0;
    return (int32_t)f;
}

/* ------------------------------------------------------------------ */
/* Sec. III.C's lossy membership test (the byte map)                    */
/* ------------------------------------------------------------------ */
/* A byte map of s = 2^b entries marks, for every edge (i, j), the address
 *   hash(i', j') = ((i' * n + j') * 1103515245) & (s - 1)
 * computed in 32-bit arithmetic with wrap-around (as printed), on the names
 * i' = pi(i), j' = pi(j) of the current random renaming.  A draw is taken
 * for an edge when its address is marked: no edge is missed, a non-edge
 * whose address collides with an edge's is rejected like an edge.
 * Renaming (redrawn every `rename_every` sample epochs, period
 * r = epoch / rename_every, r = 0 throughout when rename_every = 0):
 * pi(v) = (a v + b) mod n with a = 1 + (w0 mod (n-1)) stepped up to the next
 * value coprime to n and b = w1 mod n, (w0, w1) the first two words of
 * Philox counter (r, 0, 0, 0x09000000). */
typedef struct {
    uint8_t* map;
    uint32_t mask, n, a, b;
    int32_t period;
} orc_bytemap;

static uint32_t gcd_u32(uint32_t x, uint32_t y) {
    while (y) { uint32_t t = x % y; x = y; y = t; }
    return x;
}

static void bytemap_perm(uint64_t seed, int32_t period, uint32_t n, uint32_t* a, uint32_t* b) {
    uint32_t w0 = philox_word(seed, (uint32_t)period, 0u, 0u, 0x09000000u, 0);
    uint32_t w1 = philox_word(seed, (uint32_t)period, 0u, 0u, 0x09000000u, 1);
    uint32_t aa = 1u + (n > 1 ? w0 % (n - 1) : 0u);
    while (gcd_u32(aa, n) != 1u) aa = (aa + 1u >= n) ? 1u : aa + 1u;
    *a = aa;
    *b = w1 % n;
}

static uint32_t bytemap_name(const orc_bytemap* m, uint32_t v) {
    return (uint32_t)(((uint64_t)m->a * v + m->b) % m->n);
}

static uint32_t bytemap_addr(const orc_bytemap* m, uint32_t i, uint32_t j) {
    uint32_t ii = bytemap_name(m, i), jj = bytemap_name(m, j);
    return ((ii * m->n + jj) * 1103515245u) & m->mask;
}

/* (Re)build the map for the renaming of `period`. */
static void bytemap_build(orc_bytemap* m, const int32_t* row_ptr, const int32_t* col_idx, int32_t n,
                          uint64_t seed, int32_t period) {
    memset(m->map, 0, (size_t)m->mask + 1);
    m->n = (uint32_t)n;
    bytemap_perm(seed, period, (uint32_t)n, &m->a, &m->b);
    m->period = period;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            m->map[bytemap_addr(m, (uint32_t)i, (uint32_t)col_idx[e])] = 1;
}

/* Membership as the sampler sees it: exact (m == NULL) or the byte map. */
static int sampler_is_edge(const orc_bytemap* m, const int32_t* row_ptr, const int32_t* col_idx, int32_t i,
                           int32_t g, int64_t* false_pos) {
    if (!m) return orc_is_edge(row_ptr, col_idx, i, g);
    int marked = m->map[bytemap_addr(m, (uint32_t)i, (uint32_t)g)] != 0;
    if (marked && false_pos && !orc_is_edge(row_ptr, col_idx, i, g)) ++*false_pos;
    return marked;
}

/* Accepted non-edge partners of vertex i for sample slots t = 0..k-1
 * (g or -1 when all attempts hit an edge or i itself); bm: NULL for the
 * exact membership test, else the byte map. */
static void sample_vertex_bm(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int32_t i,
                             int32_t epoch, uint64_t seed, uint32_t tag, int32_t k, int32_t max_retries,
                             const orc_bytemap* bm, int32_t* out, int64_t* rejected, int64_t* exhausted,
                             int64_t* false_pos, int32_t rng) {
    for (int32_t t = 0; t < k; ++t) {
        int32_t got = -1;
        uint32_t state = rng ? philox_word(seed, (uint32_t)i, (uint32_t)epoch, (uint32_t)t >> 2, 0x08000000u, t & 3) : 0u;
        for (int32_t a = 0; a < max_retries; ++a) {
            int32_t g;
            if (rng) {
                state = lcg_next(state);
                g = lcg_vertex(state, n);
            } else {
                uint32_t r = philox_word(seed, (uint32_t)i, (uint32_t)epoch, (uint32_t)t >> 2, tag | (uint32_t)a, t & 3);
                g = (int32_t)draw_vertex(r, (uint32_t)n);
            }
            if (g != i && !sampler_is_edge(bm, row_ptr, col_idx, i, g, false_pos)) { got = g; break; }
            if (rejected) ++*rejected;
        }
        if (got < 0 && exhausted) ++*exhausted;
        out[t] = got;
    }
}

static void sample_vertex(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int32_t i,
                          int32_t epoch, uint64_t seed, uint32_t tag, int32_t k, int32_t max_retries,
                          int32_t* out, int64_t* rejected, int64_t* exhausted) {
    sample_vertex_bm(row_ptr, col_idx, n, i, epoch, seed, tag, k, max_retries, NULL, out, rejected, exhausted,
                     NULL, 0);
}

/* Byte-map addresses of pairs under the renaming of `period` (inspection). */
void orc_bytemap_addr(int32_t n, uint64_t seed, int32_t period, int32_t log2_size, const int32_t* pairs,
                      int64_t count, uint32_t* out, uint32_t* perm_ab) {
    orc_bytemap m;
    m.map = NULL;
    m.mask = (uint32_t)((1ull << log2_size) - 1ull);
    m.n = (uint32_t)n;
    bytemap_perm(seed, period, (uint32_t)n, &m.a, &m.b);
    if (perm_ab) { perm_ab[0] = m.a; perm_ab[1] = m.b; }
    for (int64_t q = 0; q < count; ++q) out[q] = bytemap_addr(&m, (uint32_t)pairs[2 * q], (uint32_t)pairs[2 * q + 1]);
}

/* Sec. III.C's policy: every CSR slot e = (i, j) of row i carries one
 * non-edge partner of i, drawn with counter (e>>2, epoch, 0, 0x0C000000 | a)
 * word e & 3 (e counted from the start of the graph's CSR), redrawn while it
 * hits i or an edge, at most max_retries times.  out[t]: the partner of slot
 * row_ptr[i] + t, or -1. */
static void sample_slots(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int32_t i,
                         int32_t epoch, uint64_t seed, int32_t max_retries, const orc_bytemap* bm, int32_t* out,
                         int64_t* rejected, int64_t* exhausted, int64_t* false_pos, int32_t rng) {
    for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        int32_t got = -1;
        uint32_t state = rng ? philox_word(seed, (uint32_t)e >> 2, (uint32_t)epoch, 0u, 0x07000000u, e & 3) : 0u;
        for (int32_t a = 0; a < max_retries; ++a) {
            int32_t g;
            if (rng) {
                state = lcg_next(state);
                g = lcg_vertex(state, n);
            } else {
                uint32_t r = philox_word(seed, (uint32_t)e >> 2, (uint32_t)epoch, 0u, 0x0C000000u | (uint32_t)a, e & 3);
                g = (int32_t)draw_vertex(r, (uint32_t)n);
            }
            if (g != i && !sampler_is_edge(bm, row_ptr, col_idx, i, g, false_pos)) { got = g; break; }
            if (rejected) ++*rejected;
        }
        if (got < 0 && exhausted) ++*exhausted;
        out[e - row_ptr[i]] = got;
    }
}

/* Partners of tile `tile` in block sampling (P of them, duplicates kept). */
void orc_block_partners(int32_t n, int32_t tile, int32_t epoch, uint64_t seed, int32_t P, int32_t* out) {
    for (int32_t p = 0; p < P; ++p) {
        uint32_t r = philox_word(seed, (uint32_t)tile, (uint32_t)epoch, (uint32_t)(p >> 2), 0x0D000000u, p & 3);
        out[p] = (int32_t)draw_vertex(r, (uint32_t)n);
    }
}

void orc_sample(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int32_t epoch,
                uint64_t seed, int32_t loss_stream, int32_t k, int32_t max_retries, int32_t* samples) {
    uint32_t tag = loss_stream ? 0x0E000000u : 0x0B000000u;
    for (int32_t i = 0; i < n; ++i)
        sample_vertex(row_ptr, col_idx, n, i, epoch, seed, tag, k, max_retries,
                      samples + (int64_t)i * k, NULL, NULL);
}

/* ------------------------------------------------------------------ */
/* One epoch (Fig. 4) in the per-vertex CSR form                        */
/* ------------------------------------------------------------------ */
static int epoch_range(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t d,
                       const double* x, double sigma, double mu, int32_t epoch, uint64_t seed,
                       int32_t k, int32_t max_retries, int32_t symmetric, int32_t w_formula,
                       int32_t clamp_neg_d, double z_min, int32_t B, double hist_max,
                       double* y, double* z, double* x_new, double* hist_e, double* hist_n,
                       int32_t* samples_out, int64_t* stats, double* absd,
                       int32_t block_P, int32_t block_T, int32_t* partners_out, int32_t per_slot,
                       int32_t membership, int32_t bytemap_log2, int32_t rename_every, int32_t rng,
                       int32_t a_lo, int32_t a_hi);

int orc_epoch(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t d,
              const double* x, double sigma, double mu, int32_t epoch, uint64_t seed,
              int32_t k, int32_t max_retries, int32_t symmetric, int32_t w_formula,
              int32_t clamp_neg_d, double z_min, int32_t B, double hist_max,
              double* y, double* z, double* x_new, double* hist_e, double* hist_n,
              int32_t* samples_out, int64_t* stats, double* absd,
              int32_t block_P, int32_t block_T, int32_t* partners_out, int32_t per_slot,
              int32_t membership, int32_t bytemap_log2, int32_t rename_every, int32_t rng) {
    return epoch_range(n, row_ptr, col_idx, d, x, sigma, mu, epoch, seed, k, max_retries, symmetric, w_formula,
                       clamp_neg_d, z_min, B, hist_max, y, z, x_new, hist_e, hist_n, samples_out, stats, absd,
                       block_P, block_T, partners_out, per_slot, membership, bytemap_log2, rename_every, rng, 0, n);
}

/* The terms of the anchors a_lo <= i < a_hi alone (Sec. III.E's split of
 * the numerators and denominators of Eq. 3 over workers): their edges (each
 * undirected edge's histogram entry at its smaller endpoint), their sampled
 * non-edges and, in block sampling, their rows of each tile; y, z hold the
 * sums these terms give every vertex, the histograms and counts these
 * anchors' pairs.  Summed over a partition of [0, n) they are orc_epoch's.
 * x_new is computed from these partial sums (meaningful for a_lo = 0,
 * a_hi = n only). */
int orc_epoch_range(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t d,
                    const double* x, double sigma, double mu, int32_t epoch, uint64_t seed,
                    int32_t k, int32_t max_retries, int32_t symmetric, int32_t w_formula,
                    int32_t clamp_neg_d, double z_min, int32_t B, double hist_max,
                    double* y, double* z, double* x_new, double* hist_e, double* hist_n,
                    int32_t* samples_out, int64_t* stats, double* absd,
                    int32_t block_P, int32_t block_T, int32_t* partners_out, int32_t per_slot,
                    int32_t membership, int32_t bytemap_log2, int32_t rename_every, int32_t rng,
                    int32_t a_lo, int32_t a_hi) {
    if (a_lo < 0 || a_hi > n || a_lo > a_hi) return -2;
    return epoch_range(n, row_ptr, col_idx, d, x, sigma, mu, epoch, seed, k, max_retries, symmetric, w_formula,
                       clamp_neg_d, z_min, B, hist_max, y, z, x_new, hist_e, hist_n, samples_out, stats, absd,
                       block_P, block_T, partners_out, per_slot, membership, bytemap_log2, rename_every, rng, a_lo,
                       a_hi);
}

static int epoch_range(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t d,
                       const double* x, double sigma, double mu, int32_t epoch, uint64_t seed,
                       int32_t k, int32_t max_retries, int32_t symmetric, int32_t w_formula,
                       int32_t clamp_neg_d, double z_min, int32_t B, double hist_max,
                       double* y, double* z, double* x_new, double* hist_e, double* hist_n,
                       int32_t* samples_out, int64_t* stats, double* absd,
                       int32_t block_P, int32_t block_T, int32_t* partners_out, int32_t per_slot,
                       int32_t membership, int32_t bytemap_log2, int32_t rename_every, int32_t rng,
                       int32_t a_lo, int32_t a_hi) {
    /* block sampling or the per-slot policy replace the k per-vertex samples */
    if (block_P > 0) { k = 0; per_slot = 0; }
    /* membership 1: the sampler tests pairs against the byte map of the
     * renaming period of this epoch */
    orc_bytemap bm;
    orc_bytemap* bmp = NULL;
    if (membership == 1 && block_P == 0) {
        bm.mask = (uint32_t)((1ull << bytemap_log2) - 1ull);
        bm.map = (uint8_t*)malloc((size_t)bm.mask + 1);
        if (!bm.map) return -1;
        bytemap_build(&bm, row_ptr, col_idx, n, seed, rename_every > 0 ? epoch / rename_every : 0);
        bmp = &bm;
    }
    int64_t false_pos = 0;
    int32_t smp_cap = k > 0 ? k : 1;
    if (per_slot)
        for (int32_t i = 0; i < n; ++i) smp_cap = (row_ptr[i + 1] - row_ptr[i] > smp_cap) ? row_ptr[i + 1] - row_ptr[i] : smp_cap;
    g_absd = absd;
    if (absd) memset(absd, 0, sizeof(double) * (size_t)n);
    memset(y, 0, sizeof(double) * (size_t)n * d);          /* zero numerators ... */
    memset(z, 0, sizeof(double) * (size_t)n);              /* ... and denominators */
    if (hist_e) memset(hist_e, 0, sizeof(double) * (size_t)B);
    if (hist_n) memset(hist_n, 0, sizeof(double) * (size_t)B);
    int64_t accepted = 0, rejected = 0, exhausted = 0;
    int failed = 0;
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
    /* per-thread sample buffers and counters (one set without OpenMP) */
    int32_t* smp = (int32_t*)malloc((size_t)smp_cap * sizeof(int32_t));
    int32_t* part = (int32_t*)malloc((size_t)(block_P > 0 ? block_P : 1) * sizeof(int32_t));
    int64_t acc_t = 0, rej_t = 0, exh_t = 0, fp_t = 0;
    if (!smp || !part) {
        ORC_ATOMIC failed += 1;
    }
#ifdef _OPENMP
#pragma omp barrier
#endif
    if (!failed) {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
    for (int32_t i = a_lo; i < a_hi; ++i) {
        /* edges: every CSR slot (i,j) contributes to y_i, z_i */
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            double delta = dist(x, d, i, j), dd, w;
            orc_parabola(delta, mu, sigma, 1, w_formula, clamp_neg_d, &dd, &w);
            add_wm_term(y, z, x, d, i, j, delta, dd, w);
            if (hist_e && j > i) {
                ORC_ATOMIC hist_e[hist_bin(delta, B, hist_max)] += 1.0;
            }
        }
        /* sampled non-edges anchored at i: k of them, or one per CSR slot */
        int32_t ki = k;
        if (per_slot) {
            ki = row_ptr[i + 1] - row_ptr[i];
            sample_slots(row_ptr, col_idx, n, i, epoch, seed, max_retries, bmp, smp, &rej_t, &exh_t, &fp_t, rng);
        } else {
            sample_vertex_bm(row_ptr, col_idx, n, i, epoch, seed, 0x0B000000u, k, max_retries, bmp, smp,
                             &rej_t, &exh_t, &fp_t, rng);
        }
        int32_t acc = 0;
        for (int32_t t = 0; t < ki; ++t) acc += (smp[t] >= 0);
        acc_t += acc;
        double deg = (double)(row_ptr[i + 1] - row_ptr[i]);
        double omega = acc ? ((double)n - 1.0 - deg) / (2.0 * acc) : 0.0;
        for (int32_t t = 0; t < ki; ++t) {
            if (samples_out) samples_out[per_slot ? (int64_t)row_ptr[i] + t : (int64_t)i * k + t] = smp[t];
            int32_t g = smp[t];
            if (g < 0) continue;
            double delta = dist(x, d, i, g), dd, w;
            orc_parabola(delta, mu, sigma, 0, w_formula, clamp_neg_d, &dd, &w);
            add_wm_term(y, z, x, d, i, g, delta, dd, w);
            if (symmetric) add_wm_term(y, z, x, d, g, i, delta, dd, w);
            if (hist_n) {
                ORC_ATOMIC hist_n[hist_bin(delta, B, hist_max)] += omega;
            }
        }
    }
    /* block-sampled non-edges: every vertex of a tile against the tile's partners */
    if (block_P > 0) {
        int32_t n_tiles = (n + block_T - 1) / block_T;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (int32_t tile = 0; tile < n_tiles; ++tile) {
            if ((tile + 1) * block_T <= a_lo || tile * block_T >= a_hi) continue;   /* no anchor of the range */
            orc_block_partners(n, tile, epoch, seed, block_P, part);
            if (partners_out) memcpy(partners_out + (int64_t)tile * block_P, part, sizeof(int32_t) * (size_t)block_P);
            for (int32_t i = (tile * block_T > a_lo ? tile * block_T : a_lo);
                 i < n && i < a_hi && i < (tile + 1) * block_T; ++i) {
                int32_t acc = 0;
                for (int32_t p = 0; p < block_P; ++p)
                    acc += (part[p] != i && !orc_is_edge(row_ptr, col_idx, i, part[p]));
                acc_t += acc;
                rej_t += block_P - acc;
                double deg = (double)(row_ptr[i + 1] - row_ptr[i]);
                double omega = acc ? ((double)n - 1.0 - deg) / (2.0 * acc) : 0.0;
                for (int32_t p = 0; p < block_P; ++p) {
                    int32_t g = part[p];
                    if (g == i || orc_is_edge(row_ptr, col_idx, i, g)) continue;   /* masked */
                    double delta = dist(x, d, i, g), dd, w;
                    orc_parabola(delta, mu, sigma, 0, w_formula, clamp_neg_d, &dd, &w);
                    add_wm_term(y, z, x, d, i, g, delta, dd, w);
                    if (symmetric) add_wm_term(y, z, x, d, g, i, delta, dd, w);
                    if (hist_n) {
                        ORC_ATOMIC hist_n[hist_bin(delta, B, hist_max)] += omega;
                    }
                }
            }
        }
    }
    }
    ORC_ATOMIC accepted += acc_t;
    ORC_ATOMIC rejected += rej_t;
    ORC_ATOMIC exhausted += exh_t;
    ORC_ATOMIC false_pos += fp_t;
    free(smp);
    free(part);
    }
    if (failed) {
        g_absd = NULL;
        if (bmp) free(bm.map);
        return -1;
    }
    /* x_i := y_i / z_i */
    for (int32_t i = 0; i < n; ++i)
        for (int32_t c = 0; c < d; ++c)
            x_new[(int64_t)i * d + c] = (z[i] >= z_min) ? y[(int64_t)i * d + c] / z[i]
                                                         : x[(int64_t)i * d + c];
    if (stats) {
        stats[0] = accepted;
        stats[1] = rejected;
        stats[2] = exhausted;
        stats[3] = accepted + rejected;
        stats[4] = false_pos;
    }
    g_absd = NULL;
    if (bmp) free(bm.map);
    return 0;
}

/* Edge part of Eq. 3 as the paper organises it (Fig. 4): a loop over the
 * undirected edge list, each edge updating both endpoints. */
void orc_edge_terms_edgelist(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t d,
                             const double* x, double sigma, double mu, int32_t w_formula,
                             int32_t clamp_neg_d, double* y, double* z) {
    memset(y, 0, sizeof(double) * (size_t)n * d);
    memset(z, 0, sizeof(double) * (size_t)n);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            if (j < i) continue;             /* undirected edge list: (i,j), i < j */
            double delta = dist(x, d, i, j), dd, w;
            orc_parabola(delta, mu, sigma, 1, w_formula, clamp_neg_d, &dd, &w);
            add_wm_term(y, z, x, d, i, j, delta, dd, w);
            add_wm_term(y, z, x, d, j, i, delta, dd, w);
        }
}

/* Edge part of Eq. 3 in the per-vertex CSR form used by orc_epoch. */
void orc_edge_terms_csr(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t d,
                        const double* x, double sigma, double mu, int32_t w_formula,
                        int32_t clamp_neg_d, double* y, double* z) {
    memset(y, 0, sizeof(double) * (size_t)n * d);
    memset(z, 0, sizeof(double) * (size_t)n);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            double delta = dist(x, d, i, j), dd, w;
            orc_parabola(delta, mu, sigma, 1, w_formula, clamp_neg_d, &dd, &w);
            add_wm_term(y, z, x, d, i, j, delta, dd, w);
        }
}

/* ------------------------------------------------------------------ */
/* Eq. 3 for chosen vertices only (the per-vertex view of Fig. 4)       */
/* ------------------------------------------------------------------ */
/* One pair's term (Eq. 3) added to query slot q of vertex a (partner b). */
static void add_query_term(double* y, double* z, double* absd, const double* x, int32_t d, int32_t q,
                           int64_t a, int64_t b, double delta, double dd, double w) {
    if (!(w > 0.0)) return;
    double s = (delta != 0.0) ? dd / delta : 0.0;
    for (int32_t c = 0; c < d; ++c)
        y[(int64_t)q * d + c] += w * (x[b * d + c] + s * (x[a * d + c] - x[b * d + c]));
    z[q] += w;
    absd[q] += w * fabs(s - 1.0) * delta;
}

static void query_pair(double* y, double* z, double* absd, const double* x, int32_t d, int32_t q, int64_t a,
                       int64_t b, int is_edge, double sigma, double mu, int32_t w_formula, int32_t clamp_neg_d) {
    double delta = dist(x, d, a, b), dd, w;
    orc_parabola(delta, mu, sigma, is_edge, w_formula, clamp_neg_d, &dd, &w);
    add_query_term(y, z, absd, x, d, q, a, b, delta, dd, w);
}

/* y_v, z_v and the size of the terms of y_v - z_v x_v for the n_query
 * distinct vertices query[], with the samples orc_epoch draws (exact
 * membership): Eq. 3 summed over v's edges, the non-edges sampled at v, and,
 * when symmetric, the non-edges of other anchors whose sampled partner is v
 * (Fig. 4 updates both ends of a sampled pair).  The same sums orc_epoch
 * forms for every vertex, in another order; at large n it costs one pass of
 * draws instead of every pair's arithmetic.  Returns 0, -1 when out of
 * memory, -2 for a query out of range or repeated. */
int orc_vertex_terms(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t d, const double* x,
                     double sigma, double mu, int32_t epoch, uint64_t seed, int32_t k, int32_t max_retries,
                     int32_t symmetric, int32_t w_formula, int32_t clamp_neg_d, int32_t block_P, int32_t block_T,
                     int32_t per_slot, int32_t n_query, const int32_t* query, double* y, double* z,
                     double* absd) {
    if (block_P > 0) { k = 0; per_slot = 0; }
    int32_t* qi = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t cap = k > 0 ? k : 1;
    for (int32_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] - row_ptr[i] > cap) cap = row_ptr[i + 1] - row_ptr[i];
    if (block_P > cap) cap = block_P;
    int32_t* smp = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
    if (!qi || !smp) { free(qi); free(smp); return -1; }
    for (int32_t i = 0; i < n; ++i) qi[i] = -1;
    for (int32_t q = 0; q < n_query; ++q) {
        if (query[q] < 0 || query[q] >= n || qi[query[q]] >= 0) { free(qi); free(smp); return -2; }
        qi[query[q]] = q;
    }
    memset(y, 0, sizeof(double) * (size_t)n_query * d);
    memset(z, 0, sizeof(double) * (size_t)n_query);
    memset(absd, 0, sizeof(double) * (size_t)n_query);
    /* v's edges and the non-edges anchored at v */
    for (int32_t q = 0; q < n_query; ++q) {
        int32_t v = query[q];
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
            query_pair(y, z, absd, x, d, q, v, col_idx[e], 1, sigma, mu, w_formula, clamp_neg_d);
        int32_t kv = 0;
        if (block_P > 0) {
            orc_block_partners(n, v / block_T, epoch, seed, block_P, smp);
            for (int32_t p = 0; p < block_P; ++p)
                if (smp[p] == v || orc_is_edge(row_ptr, col_idx, v, smp[p])) smp[p] = -1;   /* masked */
            kv = block_P;
        } else if (per_slot) {
            sample_slots(row_ptr, col_idx, n, v, epoch, seed, max_retries, NULL, smp, NULL, NULL, NULL, 0);
            kv = row_ptr[v + 1] - row_ptr[v];
        } else {
            sample_vertex(row_ptr, col_idx, n, v, epoch, seed, 0x0B000000u, k, max_retries, smp, NULL, NULL);
            kv = k;
        }
        for (int32_t t = 0; t < kv; ++t)
            if (smp[t] >= 0) query_pair(y, z, absd, x, d, q, v, smp[t], 0, sigma, mu, w_formula, clamp_neg_d);
    }
    /* the non-edges of every anchor i whose partner is a queried vertex */
    if (symmetric) {
        if (block_P > 0) {
            int32_t n_tiles = (n + block_T - 1) / block_T;
            for (int32_t tile = 0; tile < n_tiles; ++tile) {
                orc_block_partners(n, tile, epoch, seed, block_P, smp);
                for (int32_t p = 0; p < block_P; ++p) {
                    int32_t g = smp[p], q = qi[g];
                    if (q < 0) continue;
                    for (int32_t i = tile * block_T; i < n && i < (tile + 1) * block_T; ++i)
                        if (g != i && !orc_is_edge(row_ptr, col_idx, i, g))
                            query_pair(y, z, absd, x, d, q, g, i, 0, sigma, mu, w_formula, clamp_neg_d);
                }
            }
        } else {
            for (int32_t i = 0; i < n; ++i) {
                int32_t ki = per_slot ? row_ptr[i + 1] - row_ptr[i] : k;
                if (per_slot)
                    sample_slots(row_ptr, col_idx, n, i, epoch, seed, max_retries, NULL, smp, NULL, NULL, NULL, 0);
                else
                    sample_vertex(row_ptr, col_idx, n, i, epoch, seed, 0x0B000000u, k, max_retries, smp, NULL,
                                  NULL);
                for (int32_t t = 0; t < ki; ++t) {
                    if (smp[t] < 0 || qi[smp[t]] < 0) continue;
                    query_pair(y, z, absd, x, d, qi[smp[t]], smp[t], i, 0, sigma, mu, w_formula, clamp_neg_d);
                }
            }
        }
    }
    free(qi);
    free(smp);
    return 0;
}

/* Sum of dl over all undirected edges and over a list of sampled non-edges
 * (samples[i*k+t] = partner of anchor i, or -1). */
double orc_surrogate_L(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t d,
                       const double* x, double sigma, double mu, int32_t k, const int32_t* samples) {
    double L = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (col_idx[e] > i) L += orc_dl(dist(x, d, i, col_idx[e]), mu, sigma, 1);
        for (int32_t t = 0; t < k; ++t) {
            int32_t g = samples[(int64_t)i * k + t];
            if (g >= 0) L += orc_dl(dist(x, d, i, g), mu, sigma, 0);
        }
    }
    return L;
}

/* ------------------------------------------------------------------ */
/* Sec. III.F: slope optimisation on distance histograms                */
/* ------------------------------------------------------------------ */
/* dPE/dsigma (up to the positive factor 1/N) on histogram bins:
 * d dl+/dsigma = -u h(u) / (sigma ln2), d dl-/dsigma = u g(u) / (sigma ln2)
 * with h(u) = phi(u)/Q(u), g(u) = phi(u)/Q(-u), u = (delta-mu)/sigma. */
double orc_dpe_dsigma(const double* hist_e, const double* hist_n, int32_t B, double hist_max,
                      double mu, double sigma) {
    double bw = hist_max / (double)B, s = 0.0;
    for (int32_t b = 0; b < B; ++b) {
        if (hist_e[b] == 0.0 && hist_n[b] == 0.0) continue;
        double u = (((double)b + 0.5) * bw - mu) / sigma;
        if (hist_e[b] != 0.0) s += hist_e[b] * (-u * inv_mills(u));
        if (hist_n[b] != 0.0) s += hist_n[b] * (u * inv_mills(-u));
    }
    return s / (sigma * ORC_LN2);
}

/* Histogram entropy sum at sigma: sum_b c_e dl+(centre) + c_n dl-(centre). */
double orc_hist_pe(const double* hist_e, const double* hist_n, int32_t B, double hist_max,
                   double mu, double sigma) {
    double bw = hist_max / (double)B, s = 0.0;
    for (int32_t b = 0; b < B; ++b) {
        double c = ((double)b + 0.5) * bw;
        if (hist_e[b] != 0.0) s += hist_e[b] * orc_dl(c, mu, sigma, 1);
        if (hist_n[b] != 0.0) s += hist_n[b] * orc_dl(c, mu, sigma, 0);
    }
    return s;
}

double orc_sigma_fit(const double* hist_e, const double* hist_n, int32_t B, double hist_max,
                     double mu, double lo, double hi, int32_t iters) {
    double flo = orc_dpe_dsigma(hist_e, hist_n, B, hist_max, mu, lo);
    double fhi = orc_dpe_dsigma(hist_e, hist_n, B, hist_max, mu, hi);
    if ((flo > 0.0) == (fhi > 0.0))
        return (flo > 0.0) ? lo : hi;   /* monotone on the bracket: its lower-entropy end */
    int lo_pos = flo > 0.0;
    for (int32_t it = 0; it < iters; ++it) {
        double mid = sqrt(lo * hi);
        double fm = orc_dpe_dsigma(hist_e, hist_n, B, hist_max, mu, mid);
        if ((fm > 0.0) == lo_pos) lo = mid; else hi = mid;
    }
    return sqrt(lo * hi);
}

/* ------------------------------------------------------------------ */
/* Eq. 2: predictive entropy                                            */
/* ------------------------------------------------------------------ */
double orc_loss_exact(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t d,
                      const double* x, double sigma, double mu) {
    double N = 0.5 * (double)n * ((double)n - 1.0), s = 0.0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = i + 1; j < n; ++j)
            s += orc_dl(dist(x, d, i, j), mu, sigma, orc_is_edge(row_ptr, col_idx, i, j));
    return s / N;
}

/* dPE/dsigma over all n(n-1)/2 pairs (Eq. 2 differentiated in sigma, mu
 * fixed), up to the positive factor 1/N: the exact counterpart of
 * orc_dpe_dsigma, with each pair at its own distance instead of a bin centre. */
double orc_dpe_dsigma_exact(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t d,
                            const double* x, double mu, double sigma) {
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = i + 1; j < n; ++j) {
            double u = (dist(x, d, i, j) - mu) / sigma;
            s += orc_is_edge(row_ptr, col_idx, i, j) ? -u * inv_mills(u) : u * inv_mills(-u);
        }
    return s / (sigma * ORC_LN2);
}

/* The slope minimising Eq. 2 exactly (mu fixed): the zero of the exact
 * dPE/dsigma, by the bisection of Sec. III.F in log sigma on [lo, hi];
 * without a sign change, the bracket end with the lower entropy. */
double orc_sigma_fit_exact(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t d,
                           const double* x, double mu, double lo, double hi, int32_t iters) {
    double flo = orc_dpe_dsigma_exact(n, row_ptr, col_idx, d, x, mu, lo);
    double fhi = orc_dpe_dsigma_exact(n, row_ptr, col_idx, d, x, mu, hi);
    if ((flo > 0.0) == (fhi > 0.0)) return (flo > 0.0) ? lo : hi;
    int lo_pos = flo > 0.0;
    for (int32_t it = 0; it < iters; ++it) {
        double mid = sqrt(lo * hi);
        double fm = orc_dpe_dsigma_exact(n, row_ptr, col_idx, d, x, mu, mid);
        if ((fm > 0.0) == lo_pos) lo = mid; else hi = mid;
    }
    return sqrt(lo * hi);
}

double orc_loss_sampled(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t d,
                        const double* x, double sigma, double mu, int32_t epoch, uint64_t seed,
                        int32_t k, int32_t max_retries) {
    double N = 0.5 * (double)n * ((double)n - 1.0), s = 0.0;
    int32_t* smp = (int32_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
    if (!smp) return NAN;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (col_idx[e] > i) s += orc_dl(dist(x, d, i, col_idx[e]), mu, sigma, 1);
        sample_vertex(row_ptr, col_idx, n, i, epoch, seed, 0x0E000000u, k, max_retries, smp, NULL, NULL);
        int32_t acc = 0;
        for (int32_t t = 0; t < k; ++t) acc += (smp[t] >= 0);
        if (!acc) continue;
        double omega = ((double)n - 1.0 - (double)(row_ptr[i + 1] - row_ptr[i])) / (2.0 * acc);
        for (int32_t t = 0; t < k; ++t)
            if (smp[t] >= 0) s += omega * orc_dl(dist(x, d, i, smp[t]), mu, sigma, 0);
    }
    free(smp);
    return s / N;
}

/* Sec. III.F's second way to collect the slope histograms: in a separate
 * step, all edges (once each) and k fresh non-edge samples per vertex
 * (stream 0x0F000000, the same per-vertex draw as the epoch's samples)
 * binned at the given positions, a sample anchored at i weighing
 * (n-1-deg_i)/(2 accepted_i). */
int orc_hist_pass(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t d, const double* x,
                  int32_t epoch, uint64_t seed, int32_t k, int32_t max_retries, int32_t B, double hist_max,
                  double* hist_e, double* hist_n) {
    int32_t* smp = (int32_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
    if (!smp) return -1;
    memset(hist_e, 0, sizeof(double) * (size_t)B);
    memset(hist_n, 0, sizeof(double) * (size_t)B);
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (col_idx[e] > i) hist_e[hist_bin(dist(x, d, i, col_idx[e]), B, hist_max)] += 1.0;
        sample_vertex(row_ptr, col_idx, n, i, epoch, seed, 0x0F000000u, k, max_retries, smp, NULL, NULL);
        int32_t acc = 0;
        for (int32_t t = 0; t < k; ++t) acc += (smp[t] >= 0);
        if (!acc) continue;
        double omega = ((double)n - 1.0 - (double)(row_ptr[i + 1] - row_ptr[i])) / (2.0 * acc);
        for (int32_t t = 0; t < k; ++t)
            if (smp[t] >= 0) hist_n[hist_bin(dist(x, d, i, smp[t]), B, hist_max)] += omega;
    }
    free(smp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Full run: Fig. 4 repeated for a fixed number of epochs               */
/* ------------------------------------------------------------------ */
int orc_run(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t d,
            double* x, double* sigma, double mu, int32_t epoch0, int32_t epochs, uint64_t seed,
            int32_t k, int32_t max_retries, int32_t symmetric, int32_t w_formula, int32_t clamp_neg_d,
            double z_min, int32_t B, double hist_max, int32_t sigma_every, int64_t* stats,
            int32_t block_P, int32_t block_T, int32_t per_slot, int32_t sigma_source, int32_t membership,
            int32_t bytemap_log2, int32_t rename_every, int32_t rng) {
    size_t nd = (size_t)n * d;
    double* y = (double*)malloc(nd * sizeof(double));
    double* z = (double*)malloc((size_t)n * sizeof(double));
    double* xn = (double*)malloc(nd * sizeof(double));
    double* he = (double*)malloc((size_t)B * sizeof(double));
    double* hn = (double*)malloc((size_t)B * sizeof(double));
    if (!y || !z || !xn || !he || !hn) { free(y); free(z); free(xn); free(he); free(hn); return -1; }
    int64_t st[5];
    if (stats) memset(stats, 0, 5 * sizeof(int64_t));
    for (int32_t e = 0; e < epochs; ++e) {
        int32_t ep = epoch0 + e;
        orc_epoch(n, row_ptr, col_idx, d, x, *sigma, mu, ep, seed, k, max_retries, symmetric,
                  w_formula, clamp_neg_d, z_min, B, hist_max, y, z, xn, he, hn, NULL, st, NULL,
                  block_P, block_T, NULL, per_slot, membership, bytemap_log2, rename_every, rng);
        memcpy(x, xn, nd * sizeof(double));
        if (sigma_every > 0 && ((ep + 1) % sigma_every) == 0) {
            /* sigma_source 1: histograms of a separate pass at the new positions */
            if (sigma_source == 1 &&
                orc_hist_pass(n, row_ptr, col_idx, d, x, ep, seed, k, max_retries, B, hist_max, he, hn) != 0)
                break;
            *sigma = orc_sigma_fit(he, hn, B, hist_max, mu, 1e-3, 1e3, 60);
        }
        if (stats) for (int q = 0; q < 5; ++q) stats[q] += st[q];
    }
    free(y); free(z); free(xn); free(he); free(hn);
    return 0;
}
