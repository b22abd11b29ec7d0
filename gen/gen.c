/*
 * Seeded synthetic graph generators.
 *
 * This file is the input side shared by the GPU engine's tests/benchmarks and
 * by the CPU oracle's tests. It holds no clique arithmetic: it only draws
 * random graphs and writes them out as canonical CSR (rows sorted ascending,
 * symmetric, no self-loops, no duplicate edges, int32 ids and offsets).
 *
 * Determinism across machines (x86-64 here, aarch64 on the GPU host): all
 * randomness is integer (SplitMix64 seeding + xoshiro256**, both public
 * algorithms by Blackman and Vigna), and the few real-valued steps use only
 * IEEE-754 +,-,*,/ (the library is built with -ffp-contract=off so no fused
 * multiply-add changes a rounding) through gen_log/gen_exp below, which are
 * written here from their series definitions instead of calling libm, whose
 * last-bit behaviour differs between platforms.
 *
 * Graph families (the workloads the paper's evaluation graphs are shaped
 * like, Table I: power-law social/web graphs, plus closed-form checks):
 *   gen_er       G(n, m): uniform pairs without duplicates or self-loops.
 *   gen_chunglu  Chung-Lu expected-degree graph, power-law weights, capped,
 *                plus planted cliques (Miller-Hagberg O(n+m) edge skipping).
 *   gen_rmat     R-MAT (Chakrabarti-Zhan-Faloutsos) edge sampling.
 *   gen_batch    many G(n, p) graphs of power-law sizes, one in eight joined
 *                (disjoint union) with a Moon-Moser K_{3,...,3} block.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ PRNG */

static uint64_t sm64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } rng_t;

static void rng_seed(rng_t *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; i++) r->s[i] = sm64_next(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t out = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

/* uniform double in (0, 1] (never 0, so its log is finite) */
static inline double rng_unit_open0(rng_t *r) {
    return (double)((rng_next(r) >> 11) + 1) * (1.0 / 9007199254740992.0);
}

/* uniform double in [0, 1) */
static inline double rng_unit(rng_t *r) {
    return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0);
}

/* uniform integer in [0, n), unbiased (Lemire's multiply-shift with rejection) */
static uint64_t rng_below(rng_t *r, uint64_t n) {
    if (n <= 1) return 0;
    for (;;) {
        uint64_t x = rng_next(r);
        __uint128_t m = (__uint128_t)x * n;
        uint64_t lo = (uint64_t)m;
        if (lo >= n) return (uint64_t)(m >> 64);
        uint64_t thresh = (0 - n) % n;
        if (lo >= thresh) return (uint64_t)(m >> 64);
    }
}

/* ------------------------------------------- portable real-valued helpers */

static const double LN2 = 0.69314718055994530942;

/* natural log for x > 0: x = f * 2^e with f in [sqrt(1/2), sqrt(2)),
 * log f = 2 atanh(s), s = (f-1)/(f+1), |s| < 0.1716, odd series to s^41. */
static double gen_log(double x) {
    int e = 0;
    double f = x;
    while (f >= 1.4142135623730951) { f *= 0.5; e++; }
    while (f < 0.7071067811865476) { f *= 2.0; e--; }
    double s = (f - 1.0) / (f + 1.0);
    double s2 = s * s, term = s, sum = 0.0;
    for (int k = 1; k <= 41; k += 2) {
        sum += term / (double)k;
        term *= s2;
    }
    return 2.0 * sum + (double)e * LN2;
}

/* exp(x): x = k ln2 + r, |r| <= ln2/2, Taylor series to r^24, scale by 2^k */
static double gen_exp(double x) {
    double kf = x / LN2;
    long k = (long)(kf < 0 ? kf - 0.5 : kf + 0.5);
    double r = x - (double)k * LN2;
    double term = 1.0, sum = 1.0;
    for (int i = 1; i <= 24; i++) {
        term *= r / (double)i;
        sum += term;
    }
    while (k > 0) { sum *= 2.0; k--; }
    while (k < 0) { sum *= 0.5; k++; }
    return sum;
}

static double gen_pow(double b, double y) { return gen_exp(y * gen_log(b)); }

/* floor for values well inside int64 range */
static int64_t gen_floor(double x) {
    int64_t i = (int64_t)x;
    if ((double)i > x) i--;
    return i;
}

/* --------------------------------------------------- edge list -> CSR */

typedef struct {
    int32_t *u, *v;
    int64_t len, cap;
} edges_t;

static int edges_push(edges_t *e, int32_t a, int32_t b) {
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
    e->u[e->len] = a;
    e->v[e->len] = b;
    e->len++;
    return 0;
}

static void edges_free(edges_t *e) {
    free(e->u);
    free(e->v);
    memset(e, 0, sizeof(*e));
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void sort_row(int32_t *p, int64_t len) {
    if (len < 24) {
        for (int64_t i = 1; i < len; i++) {
            int32_t key = p[i];
            int64_t j = i - 1;
            while (j >= 0 && p[j] > key) { p[j + 1] = p[j]; j--; }
            p[j + 1] = key;
        }
    } else {
        qsort(p, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

/*
 * Canonicalise an undirected edge list over n vertices: drop self-loops,
 * symmetrise, sort rows, remove duplicates. Writes *row_ptr (n+1 int32) and
 * *col (row_ptr[n] int32), both malloc'd; the caller frees them with gen_free.
 * Returns 0, or -1 on allocation failure / int32 overflow.
 */
static int edges_to_csr(const edges_t *e, int32_t n, int32_t **row_ptr_out, int32_t **col_out) {
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t i = 0; i < e->len; i++) {
        if (e->u[i] == e->v[i]) continue;
        cnt[e->u[i] + 1]++;
        cnt[e->v[i] + 1]++;
    }
    for (int32_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    int64_t total = cnt[n];
    int32_t *tmp = (int32_t *)malloc((size_t)(total ? total : 1) * sizeof(int32_t));
    int64_t *pos = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    if (!tmp || !pos) { free(cnt); free(tmp); free(pos); return -1; }
    for (int32_t i = 0; i < n; i++) pos[i] = cnt[i];
    for (int64_t i = 0; i < e->len; i++) {
        int32_t a = e->u[i], b = e->v[i];
        if (a == b) continue;
        tmp[pos[a]++] = b;
        tmp[pos[b]++] = a;
    }
    /* sort + dedupe each row in place; pos[i] becomes the unique count */
#pragma omp parallel for schedule(dynamic, 256)
    for (int32_t i = 0; i < n; i++) {
        int32_t *p = tmp + cnt[i];
        int64_t len = cnt[i + 1] - cnt[i];
        sort_row(p, len);
        int64_t w = 0;
        for (int64_t j = 0; j < len; j++)
            if (w == 0 || p[w - 1] != p[j]) p[w++] = p[j];
        pos[i] = w;
    }
    int64_t m2 = 0;
    for (int32_t i = 0; i < n; i++) m2 += pos[i];
    if (m2 > INT32_MAX) { free(cnt); free(tmp); free(pos); return -1; }
    int32_t *rp = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *col = (int32_t *)malloc((size_t)(m2 ? m2 : 1) * sizeof(int32_t));
    if (!rp || !col) { free(cnt); free(tmp); free(pos); free(rp); free(col); return -1; }
    rp[0] = 0;
    for (int32_t i = 0; i < n; i++) rp[i + 1] = rp[i] + (int32_t)pos[i];
#pragma omp parallel for schedule(dynamic, 256)
    for (int32_t i = 0; i < n; i++)
        memcpy(col + rp[i], tmp + cnt[i], (size_t)pos[i] * sizeof(int32_t));
    free(cnt);
    free(tmp);
    free(pos);
    *row_ptr_out = rp;
    *col_out = col;
    return 0;
}

void gen_free(void *p) { free(p); }

/* ------------------------------------------------------------ G(n, m) */

/*
 * Erdos-Renyi G(n, m): draw ordered pairs (u, v) uniformly, reject u == v and
 * pairs already drawn (as unordered edges), until m distinct edges exist.
 */
int gen_er(int32_t n, int64_t m, uint64_t seed, int32_t **row_ptr, int32_t **col) {
    if (n < 0 || m < 0 || (n < 2 && m > 0)) return -1;
    if ((double)m > 0.5 * (double)n * (double)(n - 1)) return -1;
    rng_t r;
    rng_seed(&r, seed);
    /* open-addressing set of accepted edges, key = (min << 32) | max */
    uint64_t cap = 16;
    while (cap < (uint64_t)(m * 2 + 16)) cap <<= 1;
    uint64_t *set = (uint64_t *)malloc(cap * sizeof(uint64_t));
    if (!set) return -1;
    memset(set, 0xff, cap * sizeof(uint64_t));
    edges_t e = {0};
    int64_t have = 0;
    while (have < m) {
        int32_t a = (int32_t)rng_below(&r, (uint64_t)n);
        int32_t b = (int32_t)rng_below(&r, (uint64_t)n);
        if (a == b) continue;
        uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a);
        uint64_t key = (lo << 32) | hi;
        uint64_t h = key * 0x9E3779B97F4A7C15ull;
        uint64_t slot = (h >> 20) & (cap - 1);
        int dup = 0;
        while (set[slot] != ~0ull) {
            if (set[slot] == key) { dup = 1; break; }
            slot = (slot + 1) & (cap - 1);
        }
        if (dup) continue;
        set[slot] = key;
        if (edges_push(&e, a, b)) { free(set); edges_free(&e); return -1; }
        have++;
    }
    free(set);
    int rc = edges_to_csr(&e, n, row_ptr, col);
    edges_free(&e);
    return rc;
}

/* ---------------------------------------------------------- Chung-Lu */

/* w_i = min(cap, c * (i+1)^(-1/(gamma-1))): mean weight for a given c */
static double cl_mean(double c, int32_t n, double expo, double wcap, const double *base) {
    double s = 0.0;
    for (int32_t i = 0; i < n; i++) {
        double w = c * base[i];
        s += (w < wcap ? w : wcap);
    }
    (void)expo;
    return s / (double)n;
}

/*
 * Chung-Lu expected-degree graph with planted cliques.
 *   weights: w_i = min(wcap, c (i+1)^(-1/(gamma-1))), c chosen by bisection
 *            so that the mean of the capped weights equals mean_deg;
 *   edges:   each pair {i, j} independently with probability
 *            min(1, w_i w_j / sum(w)), drawn with the Miller-Hagberg skip
 *            method (weights are non-increasing in i, as it requires);
 *   planted: n_planted cliques, sizes uniform in [kmin, kmax], each on
 *            vertices drawn uniformly without replacement (cliques may
 *            overlap one another).
 */
int gen_chunglu(int32_t n, double mean_deg, double gamma, double wcap, int32_t n_planted,
                int32_t kmin, int32_t kmax, uint64_t seed, int32_t **row_ptr, int32_t **col) {
    if (n < 2 || gamma <= 1.0 || mean_deg <= 0 || kmin < 0 || kmax < kmin || kmax > n) return -1;
    rng_t r;
    rng_seed(&r, seed);
    double expo = -1.0 / (gamma - 1.0);
    double *base = (double *)malloc((size_t)n * sizeof(double));
    double *w = (double *)malloc((size_t)n * sizeof(double));
    if (!base || !w) { free(base); free(w); return -1; }
    for (int32_t i = 0; i < n; i++) base[i] = gen_pow((double)(i + 1), expo);
    double lo = 0.0, hi = 1.0;
    while (cl_mean(hi, n, expo, wcap, base) < mean_deg) hi *= 2.0;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (cl_mean(mid, n, expo, wcap, base) < mean_deg) lo = mid; else hi = mid;
    }
    double c = 0.5 * (lo + hi), S = 0.0;
    for (int32_t i = 0; i < n; i++) {
        double x = c * base[i];
        w[i] = x < wcap ? x : wcap;
        S += w[i];
    }
    free(base);
    edges_t e = {0};
    for (int32_t u = 0; u + 1 < n; u++) {
        int64_t v = u + 1;
        double p = w[u] * w[v] / S;
        if (p > 1.0) p = 1.0;
        while (v < n && p > 0.0) {
            if (p != 1.0) {
                double rr = rng_unit_open0(&r);
                v += gen_floor(gen_log(rr) / gen_log(1.0 - p));
            }
            if (v < n) {
                double q = w[u] * w[v] / S;
                if (q > 1.0) q = 1.0;
                double rr = rng_unit(&r);
                if (rr < q / p) {
                    if (edges_push(&e, u, (int32_t)v)) { free(w); edges_free(&e); return -1; }
                }
                p = q;
                v += 1;
            }
        }
    }
    free(w);
    int32_t *pick = (int32_t *)malloc((size_t)(kmax > 0 ? kmax : 1) * sizeof(int32_t));
    if (!pick) { edges_free(&e); return -1; }
    for (int32_t t = 0; t < n_planted; t++) {
        int32_t k = kmin + (int32_t)rng_below(&r, (uint64_t)(kmax - kmin + 1));
        int32_t got = 0;
        while (got < k) {
            int32_t cand = (int32_t)rng_below(&r, (uint64_t)n);
            int dup = 0;
            for (int32_t j = 0; j < got; j++)
                if (pick[j] == cand) { dup = 1; break; }
            if (!dup) pick[got++] = cand;
        }
        for (int32_t a = 0; a < k; a++)
            for (int32_t b = a + 1; b < k; b++)
                if (edges_push(&e, pick[a], pick[b])) { free(pick); edges_free(&e); return -1; }
    }
    free(pick);
    int rc = edges_to_csr(&e, n, row_ptr, col);
    edges_free(&e);
    return rc;
}

/* -------------------------------------------------------------- R-MAT */

/*
 * R-MAT: edge_factor * 2^scale samples; each sample picks one of four
 * quadrants per level with probabilities (a, b, c, 1-a-b-c), quantised to
 * 16 bits (one 64-bit draw serves four levels). Quadrant b sets the column
 * bit, c the row bit, d both. No noise and no vertex permutation. Samples are
 * split into chunks of 2^20, chunk j drawing from its own stream seeded with
 * SplitMix64(seed, j), so the output does not depend on the thread count.
 * Self-loops are dropped and the result symmetrised and deduplicated.
 */
int gen_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c, uint64_t seed,
             int32_t **row_ptr, int32_t **col) {
    if (scale < 1 || scale > 30 || edge_factor < 0 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0)
        return -1;
    int32_t n = (int32_t)1 << scale;
    int64_t ns = (int64_t)edge_factor << scale;
    uint32_t ta = (uint32_t)gen_floor(a * 65536.0 + 0.5);
    uint32_t tb = ta + (uint32_t)gen_floor(b * 65536.0 + 0.5);
    uint32_t tc = tb + (uint32_t)gen_floor(c * 65536.0 + 0.5);
    edges_t e = {0};
    e.u = (int32_t *)malloc((size_t)(ns ? ns : 1) * sizeof(int32_t));
    e.v = (int32_t *)malloc((size_t)(ns ? ns : 1) * sizeof(int32_t));
    if (!e.u || !e.v) { edges_free(&e); return -1; }
    e.len = e.cap = ns;
    const int64_t CH = (int64_t)1 << 20;
    int64_t nch = (ns + CH - 1) / CH;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < nch; ch++) {
        uint64_t sx = seed ^ ((uint64_t)ch * 0xD1B54A32D192ED03ull);
        rng_t r;
        rng_seed(&r, sm64_next(&sx));
        int64_t lo = ch * CH, hi = lo + CH < ns ? lo + CH : ns;
        for (int64_t i = lo; i < hi; i++) {
            uint32_t ru = 0, rv = 0;
            uint64_t bits = 0;
            for (int32_t l = 0; l < scale; l++) {
                if ((l & 3) == 0) bits = rng_next(&r);
                uint32_t x = (uint32_t)(bits & 0xffff);
                bits >>= 16;
                uint32_t rowb = 0, colb = 0;
                if (x < ta) {
                } else if (x < tb) {
                    colb = 1;
                } else if (x < tc) {
                    rowb = 1;
                } else {
                    rowb = 1;
                    colb = 1;
                }
                ru |= rowb << (scale - 1 - l);
                rv |= colb << (scale - 1 - l);
            }
            e.u[i] = (int32_t)ru;
            e.v[i] = (int32_t)rv;
        }
    }
    int rc = edges_to_csr(&e, n, row_ptr, col);
    edges_free(&e);
    return rc;
}

/* ------------------------------------------------------------ batched */

/*
 * G graphs concatenated into one CSR. Graph g has vertex ids
 * [graph_ptr[g], graph_ptr[g+1]). Its G(n, p) part has n drawn from the
 * continuous power law density proportional to n^-alpha on [nmin, nmax]
 * (inverse CDF, rounded to nearest), mean degree D uniform in [dmin, dmax],
 * p = min(1, D/(n-1)), edges by Batagelj-Brandes geometric skipping. When
 * g % mm_every == 0 a Moon-Moser block (complete multipartite graph with
 * parts of size 3) on n_MM in {15, 30, 45} new vertices is appended,
 * disjoint from the G(n, p) part. mm_sizes_out[g] receives n_MM (0 if none).
 * Writes *graph_ptr (G+1), *row_ptr, *col; free with gen_free.
 */
int gen_batch(int32_t G, double nmin, double nmax, double alpha, double dmin, double dmax,
              int32_t mm_every, uint64_t seed, int32_t **graph_ptr, int32_t **row_ptr,
              int32_t **col, int32_t *mm_sizes_out) {
    if (G <= 0 || nmin < 2 || nmax < nmin || alpha <= 1.0 || mm_every <= 0) return -1;
    rng_t r;
    rng_seed(&r, seed);
    int32_t *gp = (int32_t *)malloc(((size_t)G + 1) * sizeof(int32_t));
    if (!gp) return -1;
    edges_t e = {0};
    int64_t off = 0;
    gp[0] = 0;
    double a1 = 1.0 - alpha;
    double lo_t = gen_pow(nmin, a1), hi_t = gen_pow(nmax, a1);
    for (int32_t g = 0; g < G; g++) {
        double u = rng_unit(&r);
        double nreal = gen_pow(lo_t + u * (hi_t - lo_t), 1.0 / a1);
        int32_t n = (int32_t)gen_floor(nreal + 0.5);
        if (n < (int32_t)nmin) n = (int32_t)nmin;
        if (n > (int32_t)nmax) n = (int32_t)nmax;
        double D = dmin + rng_unit(&r) * (dmax - dmin);
        double p = D / (double)(n - 1);
        if (p > 1.0) p = 1.0;
        int32_t base = (int32_t)off;
        if (p >= 1.0) {
            for (int32_t x = 0; x < n; x++)
                for (int32_t y = x + 1; y < n; y++)
                    if (edges_push(&e, base + x, base + y)) goto fail;
        } else {
            double lq = gen_log(1.0 - p);
            int64_t v = 1, w = -1;
            while (v < n) {
                double rr = rng_unit_open0(&r);
                w = w + 1 + gen_floor(gen_log(rr) / lq);
                while (w >= v && v < n) { w -= v; v++; }
                if (v < n)
                    if (edges_push(&e, base + (int32_t)v, base + (int32_t)w)) goto fail;
            }
        }
        int32_t nmm = 0;
        if (g % mm_every == 0) {
            nmm = 15 * (1 + (int32_t)rng_below(&r, 3));
            int32_t mb = base + n;
            for (int32_t x = 0; x < nmm; x++)
                for (int32_t y = x + 1; y < nmm; y++)
                    if (x / 3 != y / 3)
                        if (edges_push(&e, mb + x, mb + y)) goto fail;
        }
        if (mm_sizes_out) mm_sizes_out[g] = nmm;
        off += n + nmm;
        if (off > INT32_MAX) goto fail;
        gp[g + 1] = (int32_t)off;
    }
    {
        int rc = edges_to_csr(&e, (int32_t)off, row_ptr, col);
        edges_free(&e);
        if (rc) { free(gp); return rc; }
        *graph_ptr = gp;
        return 0;
    }
fail:
    edges_free(&e);
    free(gp);
    return -1;
}

/* G(n, p) alone (same skipping as gen_batch), for mid-size random tests */
int gen_gnp(int32_t n, double p, uint64_t seed, int32_t **row_ptr, int32_t **col) {
    if (n < 0 || p < 0 || p > 1) return -1;
    rng_t r;
    rng_seed(&r, seed);
    edges_t e = {0};
    if (p >= 1.0) {
        for (int32_t x = 0; x < n; x++)
            for (int32_t y = x + 1; y < n; y++)
                if (edges_push(&e, x, y)) { edges_free(&e); return -1; }
    } else if (p > 0.0) {
        double lq = gen_log(1.0 - p);
        int64_t v = 1, w = -1;
        while (v < n) {
            double rr = rng_unit_open0(&r);
            w = w + 1 + gen_floor(gen_log(rr) / lq);
            while (w >= v && v < n) { w -= v; v++; }
            if (v < n)
                if (edges_push(&e, (int32_t)v, (int32_t)w)) { edges_free(&e); return -1; }
        }
    }
    int rc = edges_to_csr(&e, n, row_ptr, col);
    edges_free(&e);
    return rc;
}

/* exposed for the generator's own sanity tests */
double gen_log_for_test(double x) { return gen_log(x); }
double gen_exp_for_test(double x) { return gen_exp(x); }
