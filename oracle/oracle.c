/*
 * CPU oracle for maximal clique enumeration -- TEST INFRASTRUCTURE ONLY.
 * (See oracle.h for the definitions; only tests, the smoke check and the
 * benchmark's CPU baseline may use this code.)
 *
 * Everything is written for a reader checking it against the paper:
 * sets are sorted int arrays, adjacency is a binary search in a sorted row,
 * the recursion is a plain restatement of Bron-Kerbosch with Tomita pivoting
 * (Sec. II-B, Algorithm 2; without a pivot, Algorithm 1), and roots follow
 * Algorithm 3 over the degeneracy order. No blocking, bitsets or fusion.
 */
#include "oracle.h"

#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------- hash */

/* SplitMix64 output finaliser (Steele, Lea, Flood 2014) */
static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t oracle_clique_hash(const int32_t *ids, int32_t k) {
    uint64_t s = 0;
    for (int32_t i = 0; i < k; i++) s += mix64((uint64_t)(int64_t)ids[i] + 1ull);
    return mix64(s + (uint64_t)k * 0x9E3779B97F4A7C15ull);
}

/* -------------------------------------------------------- validation */

static int row_has(const int32_t *row, int32_t len, int32_t x) {
    int32_t lo = 0, hi = len;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (row[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo < len && row[lo] == x;
}

int oracle_validate(int32_t n, const int32_t *row_ptr, const int32_t *col) {
    if (n < 0 || !row_ptr) return 1;
    if (row_ptr[0] != 0) return 1;
    for (int32_t v = 0; v < n; v++)
        if (row_ptr[v + 1] < row_ptr[v]) return 1;
    if (row_ptr[n] % 2 != 0) return 1;
    for (int32_t v = 0; v < n; v++) {
        for (int32_t i = row_ptr[v]; i < row_ptr[v + 1]; i++) {
            int32_t u = col[i];
            if (u < 0 || u >= n || u == v) return 1;
            if (i > row_ptr[v] && col[i - 1] >= u) return 1; /* unsorted or duplicate */
        }
    }
    for (int32_t v = 0; v < n; v++)
        for (int32_t i = row_ptr[v]; i < row_ptr[v + 1]; i++) {
            int32_t u = col[i];
            if (!row_has(col + row_ptr[u], row_ptr[u + 1] - row_ptr[u], v)) return 1;
        }
    return 0;
}

/* ------------------------------------------------- degeneracy peel */

int64_t oracle_peel(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t *core,
                    int32_t *rank, int32_t *order) {
    if (n < 0) return -1;
    int32_t *deg = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    char *removed = (char *)calloc((size_t)n + 1, 1);
    int32_t *rem = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *S = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!deg || !removed || !rem || !S) {
        free(deg); free(removed); free(rem); free(S);
        return -2;
    }
    int32_t nrem = n;
    for (int32_t v = 0; v < n; v++) {
        deg[v] = row_ptr[v + 1] - row_ptr[v];
        rem[v] = v; /* remaining vertices, kept in ascending id */
    }
    int32_t k = 0, next = 0;
    int64_t rounds = 0;
    while (nrem > 0) {
        int32_t mind = deg[rem[0]];
        for (int32_t i = 1; i < nrem; i++)
            if (deg[rem[i]] < mind) mind = deg[rem[i]];
        if (mind > k) k = mind;
        /* S = remaining vertices with degree <= k, ascending id */
        int32_t ns = 0, keep = 0;
        for (int32_t i = 0; i < nrem; i++) {
            int32_t v = rem[i];
            if (deg[v] <= k) S[ns++] = v; else rem[keep++] = v;
        }
        nrem = keep;
        for (int32_t i = 0; i < ns; i++) {
            int32_t v = S[i];
            if (rank) rank[v] = next;
            if (order) order[next] = v;
            if (core) core[v] = k;
            next++;
            removed[v] = 1;
        }
        for (int32_t i = 0; i < ns; i++) {
            int32_t v = S[i];
            for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; j++)
                if (!removed[col[j]]) deg[col[j]]--;
        }
        rounds++;
    }
    free(deg); free(removed); free(rem); free(S);
    return rounds;
}

/* ------------------------------------------------ Bron-Kerbosch */

static int cmp_int32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

typedef struct {
    const int32_t *ap;    /* relabelled adjacency offsets, [n+1] */
    const int32_t *adj;   /* neighbours of rank r as sorted ranks */
    const int32_t *order; /* rank -> input id */
    int32_t mode;         /* pivot rule */
    int32_t second_level; /* one subtree per edge (Algorithm 4) */
} graph_t;

typedef struct {
    const graph_t *g;
    int32_t root;      /* rank of the current first-level subtree's vertex */
    int32_t *R;        /* current clique, ranks */
    int32_t rlen;
    int32_t *ids;      /* scratch for input ids when reporting */
    uint64_t count, hash, nodes;
    uint64_t work;     /* bitset word operations the GPU formulation needs (see bk) */
    int32_t words;     /* 32-bit words per bitset row for the current root: ceil(|P0|/32) */
    uint64_t *hist;
    int32_t hist_len, max_size;
    uint64_t node_cap;  /* 0 = none; else a root's walk stops after this many calls */
    uint64_t node_base; /* w->nodes when the current root started */
    int aborted;        /* the current root's walk hit node_cap */
} walk_t;

static int adjacent(const graph_t *g, int32_t a, int32_t b) {
    return row_has(g->adj + g->ap[a], g->ap[a + 1] - g->ap[a], b);
}

/* out = A n N(v), A sorted; returns |out| (out sorted) */
static int32_t intersect_nbrs(const graph_t *g, const int32_t *A, int32_t na, int32_t v, int32_t *out) {
    const int32_t *row = g->adj + g->ap[v];
    int32_t deg = g->ap[v + 1] - g->ap[v], k = 0;
    if (na > deg) { /* walk both sorted lists */
        int32_t i = 0, j = 0;
        while (i < na && j < deg) {
            if (A[i] < row[j]) i++;
            else if (A[i] > row[j]) j++;
            else { out[k++] = A[i]; i++; j++; }
        }
    } else {
        for (int32_t i = 0; i < na; i++)
            if (row_has(row, deg, A[i])) out[k++] = A[i];
    }
    return k;
}

static void report(walk_t *w) {
    for (int32_t i = 0; i < w->rlen; i++) w->ids[i] = w->g->order[w->R[i]];
    w->count++;
    w->hash += oracle_clique_hash(w->ids, w->rlen);
    if (w->rlen > w->max_size) w->max_size = w->rlen;
    if (w->rlen < w->hist_len) w->hist[w->rlen]++;
}

/*
 * One call of Algorithm 2 (Bron-Kerbosch with pivoting), or of Algorithm 1
 * in ORACLE_NO_PIVOT mode. X is held as two sorted lists (Sec. III-E):
 * XP = excluded vertices from the root's P (ranks > root), XX = excluded
 * vertices from the root's X (ranks < root); X = XP u XX. P and XP are owned
 * by this call and modified in place; XP has room for np more entries.
 */
static void bk(walk_t *w, int32_t *P, int32_t np, int32_t *XP, int32_t nxp, const int32_t *XX,
               int32_t nxx) {
    const graph_t *g = w->g;
    w->nodes++;
    if (w->node_cap && w->nodes - w->node_base > w->node_cap) {
        w->aborted = 1;
        return;
    }
    if (np == 0 && nxp == 0 && nxx == 0) { /* R is a maximal clique */
        report(w);
        return;
    }
    if (np == 0) return; /* X non-empty: every branch is empty */

    /* branch set B, evaluated once: P - N(pivot), or all of P (Algorithm 1) */
    int32_t *B = (int32_t *)malloc((size_t)np * sizeof(int32_t));
    int32_t nb = 0;
    if (g->mode == ORACLE_NO_PIVOT) {
        memcpy(B, P, (size_t)np * sizeof(int32_t));
        nb = np;
    } else {
        /* pivot u maximising |P n N(u)|, ties to the smallest rank. The
         * candidates are visited in ascending rank; `scanned` counts them up
         * to the first that reaches the largest possible score (|P| for an
         * excluded vertex, |P|-1 for a vertex of P), after which no later
         * candidate can win. It feeds only the work counter. */
        int32_t best = -1, best_u = -1;
        const int32_t *lists[3] = {P, XP, XX};
        int32_t lens[3] = {np, nxp, g->mode == ORACLE_PIVOT_FULL ? nxx : 0};
        int32_t pos[3] = {0, 0, 0};
        const int32_t bound = (lens[1] + lens[2] > 0) ? np : np - 1;
        int64_t scanned = 0, total = (int64_t)lens[0] + lens[1] + lens[2];
        int reached = 0;
        for (;;) {
            int32_t L = -1;
            for (int32_t q = 0; q < 3; q++)
                if (pos[q] < lens[q] && (L < 0 || lists[q][pos[q]] < lists[L][pos[L]])) L = q;
            if (L < 0) break;
            int32_t u = lists[L][pos[L]++], score = 0;
            for (int32_t j = 0; j < np; j++) score += adjacent(g, u, P[j]);
            if (!reached) scanned++;
            if (score == bound) reached = 1;
            if (score > best || (score == best && u < best_u)) { best = score; best_u = u; }
        }
        if (!reached) scanned = total;
        w->work += (uint64_t)w->words * (uint64_t)(scanned + 1);
        for (int32_t j = 0; j < np; j++)
            if (!adjacent(g, best_u, P[j])) B[nb++] = P[j];
    }

    if (g->mode != ORACLE_NO_PIVOT) w->work += 2ull * (uint64_t)w->words * (uint64_t)nb;
    for (int32_t bi = 0; bi < nb; bi++) {
        int32_t v = B[bi];
        /* child sets: P n N(v), X n N(v) */
        int32_t *cP = (int32_t *)malloc((size_t)(np + 1) * sizeof(int32_t));
        int32_t ncp = intersect_nbrs(g, P, np, v, cP);
        int32_t *cXP = (int32_t *)malloc((size_t)(nxp + ncp + 1) * sizeof(int32_t));
        int32_t ncxp = intersect_nbrs(g, XP, nxp, v, cXP);
        int32_t *cXX = (int32_t *)malloc((size_t)(nxx + 1) * sizeof(int32_t));
        int32_t ncxx = intersect_nbrs(g, XX, nxx, v, cXX);
        w->R[w->rlen++] = v;
        bk(w, cP, ncp, cXP, ncxp, cXX, ncxx);
        w->rlen--;
        free(cP);
        free(cXP);
        free(cXX);
        if (w->aborted) break;
        /* P = P - {v} */
        int32_t k = 0;
        for (int32_t j = 0; j < np; j++)
            if (P[j] != v) P[k++] = P[j];
        np = k;
        /* X = X u {v}: v comes from P, so it joins XP (kept sorted) */
        int32_t pos = nxp;
        while (pos > 0 && XP[pos - 1] > v) { XP[pos] = XP[pos - 1]; pos--; }
        XP[pos] = v;
        nxp++;
    }
    free(B);
}

/* Algorithm 3 for one vertex of rank r: P = later neighbours, X = earlier */
static void first_level(walk_t *w, int32_t r) {
    const graph_t *g = w->g;
    const int32_t *row = g->adj + g->ap[r];
    int32_t deg = g->ap[r + 1] - g->ap[r];
    int32_t split = 0;
    while (split < deg && row[split] < r) split++;
    int32_t np = deg - split;
    int32_t *P = (int32_t *)malloc((size_t)(np + 1) * sizeof(int32_t));
    int32_t *XP = (int32_t *)malloc((size_t)(np + 1) * sizeof(int32_t));
    memcpy(P, row + split, (size_t)np * sizeof(int32_t));
    w->words = (np + 31) / 32;
    w->root = r;
    w->rlen = 0;
    w->R[w->rlen++] = r;
    bk(w, P, np, XP, 0, row, split);
    free(P);
    free(XP);
}

/*
 * Algorithm 4 for the vertex of rank r: one subtree per later neighbour v_j,
 * with R = {r, v_j}, P = the common neighbours after v_j, X = the common
 * neighbours before v_j (held as XP = those after r, XX = those before r).
 * Every maximal clique with two or more vertices lies under the edge of its
 * two earliest vertices; an isolated vertex is a maximal clique of its own and
 * has no subtree. Tree nodes count the edge subtrees' nodes only.
 */
static void second_level(walk_t *w, int32_t r) {
    const graph_t *g = w->g;
    const int32_t *row = g->adj + g->ap[r];
    int32_t deg = g->ap[r + 1] - g->ap[r];
    int32_t split = 0;
    while (split < deg && row[split] < r) split++;
    const int32_t np = deg - split;
    const int32_t *later = row + split;
    w->words = (np + 31) / 32;
    w->root = r;
    w->rlen = 0;
    w->R[w->rlen++] = r;
    if (deg == 0) {
        report(w);
        return;
    }
    int32_t *P = (int32_t *)malloc((size_t)(np + 1) * sizeof(int32_t));
    int32_t *XP = (int32_t *)malloc((size_t)(np + 1) * sizeof(int32_t));
    int32_t *XX = (int32_t *)malloc((size_t)(split + 1) * sizeof(int32_t));
    for (int32_t j = 0; j < np; j++) {
        const int32_t vj = later[j];
        int32_t nP = 0, nXP = 0, nXX = 0;
        for (int32_t k = j + 1; k < np; k++)
            if (adjacent(g, vj, later[k])) P[nP++] = later[k];
        for (int32_t k = 0; k < j; k++)
            if (adjacent(g, vj, later[k])) XP[nXP++] = later[k];
        for (int32_t k = 0; k < split; k++)
            if (adjacent(g, vj, row[k])) XX[nXX++] = row[k];
        w->R[w->rlen++] = vj;
        bk(w, P, nP, XP, nXP, XX, nXX);
        w->rlen--;
    }
    free(P);
    free(XP);
    free(XX);
}

typedef struct {
    const graph_t *g;
    const int32_t *roots; /* ranks to process */
    int64_t n_roots;
    atomic_llong next;
    int32_t hist_len, max_deg;
    uint64_t *root_count, *root_hash, *root_nodes, *root_work; /* by input id */
    uint64_t node_cap; /* per root; 0 = none */
    /* merged results */
    pthread_mutex_t mu;
    uint64_t count, hash;
    uint64_t *hist;
    int32_t max_size;
    int failed;
} job_t;

static void *worker(void *arg) {
    job_t *job = (job_t *)arg;
    walk_t w;
    memset(&w, 0, sizeof(w));
    w.g = job->g;
    w.hist_len = job->hist_len;
    w.hist = (uint64_t *)calloc((size_t)(job->hist_len > 0 ? job->hist_len : 1), sizeof(uint64_t));
    w.R = (int32_t *)malloc(((size_t)job->max_deg + 2) * sizeof(int32_t));
    w.ids = (int32_t *)malloc(((size_t)job->max_deg + 2) * sizeof(int32_t));
    if (!w.hist || !w.R || !w.ids) {
        pthread_mutex_lock(&job->mu);
        job->failed = 1;
        pthread_mutex_unlock(&job->mu);
        free(w.hist); free(w.R); free(w.ids);
        return NULL;
    }
    for (;;) {
        long long i = atomic_fetch_add(&job->next, 1);
        if (i >= job->n_roots) break;
        int32_t r = job->roots[i];
        uint64_t c0 = w.count, h0 = w.hash, n0 = w.nodes, k0 = w.work;
        w.node_cap = job->node_cap;
        w.node_base = w.nodes;
        w.aborted = 0;
        if (job->g->second_level) second_level(&w, r);
        else first_level(&w, r);
        int32_t id = job->g->order[r];
        if (w.aborted) { /* over the cap: marked, and nothing of it kept */
            w.count = c0;
            w.hash = h0;
            if (job->root_nodes) job->root_nodes[id] = UINT64_MAX;
            if (job->root_count) job->root_count[id] = 0;
            if (job->root_hash) job->root_hash[id] = 0;
            continue;
        }
        if (job->root_count) job->root_count[id] = w.count - c0;
        if (job->root_hash) job->root_hash[id] = w.hash - h0;
        if (job->root_nodes) job->root_nodes[id] = w.nodes - n0;
        if (job->root_work) job->root_work[id] = w.work - k0;
    }
    pthread_mutex_lock(&job->mu);
    job->count += w.count;
    job->hash += w.hash;
    for (int32_t k = 0; k < job->hist_len; k++) job->hist[k] += w.hist[k];
    if (w.max_size > job->max_size) job->max_size = w.max_size;
    pthread_mutex_unlock(&job->mu);
    free(w.hist); free(w.R); free(w.ids);
    return NULL;
}

int32_t oracle_default_threads(void) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int32_t)c : 1;
}

static int run(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t mode, int32_t nthreads,
               const int32_t *roots_in, int64_t n_roots_in, uint64_t *count, uint64_t *hash,
               uint64_t *hist, int32_t hist_len, int32_t *max_size, uint64_t *root_count,
               uint64_t *root_hash, uint64_t *root_nodes, uint64_t *root_work, uint64_t node_cap) {
    if (oracle_validate(n, row_ptr, col)) return 1;
    const int32_t second = (mode & ORACLE_SECOND_LEVEL) != 0;
    mode &= ~ORACLE_SECOND_LEVEL;
    if (mode < 0 || mode > 2) return 1;
    int32_t *rank = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *order = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *ap = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *adj = (int32_t *)malloc(((size_t)row_ptr[n] + 1) * sizeof(int32_t));
    int32_t *roots = (int32_t *)malloc(((size_t)(roots_in ? n_roots_in : n) + 1) * sizeof(int32_t));
    int rc = 0;
    if (!rank || !order || !ap || !adj || !roots) { rc = 2; goto done; }
    if (oracle_peel(n, row_ptr, col, NULL, rank, order) < 0) { rc = 2; goto done; }
    /* relabel: row r lists rank[u] for u in N(order[r]), sorted */
    int32_t max_deg = 0;
    ap[0] = 0;
    for (int32_t r = 0; r < n; r++) {
        int32_t v = order[r], d = row_ptr[v + 1] - row_ptr[v];
        if (d > max_deg) max_deg = d;
        ap[r + 1] = ap[r] + d;
        int32_t *out = adj + ap[r];
        for (int32_t j = 0; j < d; j++) out[j] = rank[col[row_ptr[v] + j]];
        qsort(out, (size_t)d, sizeof(int32_t), cmp_int32);
    }
    int64_t n_roots;
    if (roots_in) {
        for (int64_t i = 0; i < n_roots_in; i++) {
            if (roots_in[i] < 0 || roots_in[i] >= n) { rc = 1; goto done; }
            roots[i] = rank[roots_in[i]];
        }
        n_roots = n_roots_in;
    } else {
        for (int32_t r = 0; r < n; r++) roots[r] = r;
        n_roots = n;
    }
    graph_t g = {ap, adj, order, mode, second};
    job_t job;
    memset(&job, 0, sizeof(job));
    job.g = &g;
    job.roots = roots;
    job.n_roots = n_roots;
    atomic_init(&job.next, 0);
    job.hist_len = hist_len > 0 ? hist_len : 0;
    job.max_deg = max_deg;
    job.root_count = root_count;
    job.root_hash = root_hash;
    job.root_nodes = root_nodes;
    job.root_work = root_work;
    job.node_cap = node_cap;
    job.hist = (uint64_t *)calloc((size_t)(job.hist_len > 0 ? job.hist_len : 1), sizeof(uint64_t));
    if (!job.hist) { rc = 2; goto done; }
    pthread_mutex_init(&job.mu, NULL);
    int32_t nt = nthreads > 0 ? nthreads : oracle_default_threads();
    if (nt > 1024) nt = 1024;
    pthread_t th[1024];
    int32_t started = 0;
    for (int32_t t = 0; t < nt; t++) {
        if (pthread_create(&th[t], NULL, worker, &job) != 0) break;
        started++;
    }
    if (started == 0) worker(&job);
    for (int32_t t = 0; t < started; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&job.mu);
    if (job.failed) { free(job.hist); rc = 2; goto done; }
    if (count) *count = job.count;
    if (hash) *hash = job.hash;
    if (hist) for (int32_t k = 0; k < hist_len; k++) hist[k] = job.hist[k];
    if (max_size) *max_size = job.max_size;
    if (hist_len <= job.max_size) rc = 5;
    free(job.hist);
done:
    free(rank); free(order); free(ap); free(adj); free(roots);
    return rc;
}

int oracle_mce(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t mode,
               int32_t nthreads, uint64_t *count, uint64_t *hash, uint64_t *hist,
               int32_t hist_len, int32_t *max_size, uint64_t *root_count,
               uint64_t *root_hash, uint64_t *root_nodes) {
    return run(n, row_ptr, col, mode, nthreads, NULL, 0, count, hash, hist, hist_len, max_size,
               root_count, root_hash, root_nodes, NULL, 0);
}

int oracle_mce_roots(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t mode,
                     int32_t nthreads, const int32_t *roots, int64_t n_roots, uint64_t *count,
                     uint64_t *hash, uint64_t *hist, int32_t hist_len, int32_t *max_size,
                     uint64_t *root_count, uint64_t *root_hash, uint64_t *root_nodes) {
    if (!roots || n_roots < 0) return 1;
    return run(n, row_ptr, col, mode, nthreads, roots, n_roots, count, hash, hist, hist_len,
               max_size, root_count, root_hash, root_nodes, NULL, 0);
}

int oracle_mce_work(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t mode,
                    int32_t nthreads, const int32_t *roots, int64_t n_roots, uint64_t *root_nodes,
                    uint64_t *root_work) {
    uint64_t count, hash;
    int32_t max_size;
    int rc = run(n, row_ptr, col, mode, nthreads, roots, roots ? n_roots : 0, &count, &hash, NULL, 0,
                 &max_size, NULL, NULL, root_nodes, root_work, 0);
    return rc == 5 ? 0 : rc; /* no histogram was asked for */
}

int oracle_mce_capped(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t mode, int32_t nthreads,
                      const int32_t *roots, int64_t n_roots, uint64_t node_cap, uint64_t *root_count,
                      uint64_t *root_hash, uint64_t *root_nodes) {
    uint64_t count, hash;
    int32_t max_size;
    if (!roots || n_roots < 0 || node_cap == 0) return 1;
    int rc = run(n, row_ptr, col, mode, nthreads, roots, n_roots, &count, &hash, NULL, 0, &max_size, root_count,
                 root_hash, root_nodes, NULL, node_cap);
    return rc == 5 ? 0 : rc;
}

/*
 * Maximal cliques of a complete multipartite graph whose parts are the
 * consecutive id ranges [first + i*part_size, first + (i+1)*part_size),
 * i < parts: exactly the sets holding one vertex of every part (every
 * transversal is a clique; any other clique misses a part and extends by a
 * vertex of it). Enumerates all part_size^parts of them and sums h(C).
 */
int oracle_multipartite(int32_t first, int32_t parts, int32_t part_size, uint64_t *count, uint64_t *hash) {
    if (parts < 0 || part_size < 1 || parts > 64) return 1;
    int32_t choice[64];
    uint64_t prefix[65];
    uint64_t c = 0, h = 0;
    if (parts == 0) { *count = 0; *hash = 0; return 0; }
    for (int32_t i = 0; i < parts; i++) choice[i] = 0;
    prefix[0] = 0;
    for (int32_t i = 0; i < parts; i++)
        prefix[i + 1] = prefix[i] + mix64((uint64_t)(int64_t)(first + i * part_size) + 1ull);
    for (;;) {
        c++;
        h += mix64(prefix[parts] + (uint64_t)parts * 0x9E3779B97F4A7C15ull);
        /* odometer: advance the last part first */
        int32_t i = parts - 1;
        while (i >= 0 && choice[i] == part_size - 1) i--;
        if (i < 0) break;
        choice[i]++;
        for (int32_t j = i + 1; j < parts; j++) choice[j] = 0;
        for (int32_t j = i; j < parts; j++)
            prefix[j + 1] = prefix[j] + mix64((uint64_t)(int64_t)(first + j * part_size + choice[j]) + 1ull);
    }
    *count = c;
    *hash = h;
    return 0;
}

/* ------------------------------------------ subtree size estimate */

/*
 * Knuth's estimator of the size of a backtrack tree (D. E. Knuth, "Estimating
 * the efficiency of backtrack programs", Math. Comp. 29 (1975) 121-136): walk
 * one random path down from the root, at each node taking one of its d
 * children with probability 1/d; the sum over the path's nodes of the product
 * of the degrees above each node is an unbiased estimate of the number of
 * nodes. The tree here is a first-level subtree of Algorithm 2 with the
 * oracle's pivot rule: the same pivot, branch set and branch order as bk, so
 * its node count is oracle_mce's per-root node count. The child for branch j
 * starts from P minus the branches before j and X plus them (Algorithm 2's
 * P = P - {v}, X = X u {v} after each branch), both intersected with N(v).
 * Random numbers: SplitMix64 (Steele, Lea, Flood 2014) seeded per root.
 */
typedef struct {
    const graph_t *g;
    const int32_t *roots; /* ranks */
    int64_t n_roots;
    int32_t probes, max_deg;
    uint64_t seed;
    double *mean, *var;   /* by index into roots */
    atomic_llong next;
    atomic_int failed;
} est_job_t;

static uint64_t sm64_next(uint64_t *s) {
    *s += 0x9E3779B97F4A7C15ull;
    return mix64(*s);
}

/* one path of the subtree of rank r; buffers hold max_deg + 1 ints each */
static double knuth_path(const graph_t *g, int32_t r, uint64_t *rng, int32_t *P, int32_t *XP, int32_t *XX,
                         int32_t *B, int32_t *T, int32_t *U) {
    const int32_t *row = g->adj + g->ap[r];
    int32_t deg = g->ap[r + 1] - g->ap[r], split = 0;
    while (split < deg && row[split] < r) split++;
    int32_t np = deg - split, nxp = 0, nxx = split;
    memcpy(P, row + split, (size_t)np * sizeof(int32_t));
    memcpy(XX, row, (size_t)split * sizeof(int32_t));
    double est = 0.0, weight = 1.0;
    for (;;) {
        est += weight;
        if (np == 0) break;
        /* pivot: largest |P n N(u)| over P u XP (u XX under the full rule), ties to the smallest rank */
        int32_t best = -1, best_u = -1;
        const int32_t *lists[3] = {P, XP, XX};
        int32_t lens[3] = {np, nxp, (g->mode == ORACLE_PIVOT_FULL) ? nxx : 0};
        for (int32_t q = 0; q < 3; q++)
            for (int32_t i = 0; i < lens[q]; i++) {
                int32_t u = lists[q][i], score = 0;
                for (int32_t j = 0; j < np; j++) score += adjacent(g, u, P[j]);
                if (score > best || (score == best && best_u > u)) { best = score; best_u = u; }
            }
        int32_t nb = 0;
        for (int32_t j = 0; j < np; j++)
            if (!adjacent(g, best_u, P[j])) B[nb++] = P[j];
        if (nb == 0) break;
        const int32_t pick = (int32_t)(((sm64_next(rng) >> 32) * (uint64_t)nb) >> 32);
        weight *= (double)nb;
        const int32_t v = B[pick];
        /* P' = (P - B[0..pick)) n N(v), B[0..pick) being the smallest branches */
        int32_t nt = 0, bi = 0;
        for (int32_t j = 0; j < np; j++) {
            while (bi < pick && B[bi] < P[j]) bi++;
            if (bi < pick && B[bi] == P[j]) continue;
            T[nt++] = P[j];
        }
        np = intersect_nbrs(g, T, nt, v, P);
        /* XP' = (XP u B[0..pick)) n N(v), merged in ascending rank */
        int32_t i = 0, k = 0, nu = 0;
        while (i < nxp || k < pick) {
            if (k >= pick || (i < nxp && XP[i] < B[k])) U[nu++] = XP[i++];
            else U[nu++] = B[k++];
        }
        nxp = intersect_nbrs(g, U, nu, v, XP);
        /* XX' = XX n N(v) */
        nt = intersect_nbrs(g, XX, nxx, v, T);
        memcpy(XX, T, (size_t)nt * sizeof(int32_t));
        nxx = nt;
    }
    return est;
}

static void *est_worker(void *arg) {
    est_job_t *job = (est_job_t *)arg;
    const size_t sz = ((size_t)job->max_deg + 2) * sizeof(int32_t);
    int32_t *buf = (int32_t *)malloc(6 * sz);
    if (!buf) { atomic_store(&job->failed, 1); return NULL; }
    int32_t *P = buf, *XP = P + job->max_deg + 2, *XX = XP + job->max_deg + 2, *B = XX + job->max_deg + 2,
            *T = B + job->max_deg + 2, *U = T + job->max_deg + 2;
    for (;;) {
        long long i = atomic_fetch_add(&job->next, 1);
        if (i >= job->n_roots) break;
        const int32_t r = job->roots[i];
        uint64_t rng = job->seed ^ mix64((uint64_t)(int64_t)job->g->order[r] + 1ull);
        double s = 0.0, s2 = 0.0;
        for (int32_t p = 0; p < job->probes; p++) {
            const double e = knuth_path(job->g, r, &rng, P, XP, XX, B, T, U);
            s += e;
            s2 += e * e;
        }
        const double m = s / job->probes;
        job->mean[i] = m;
        job->var[i] = job->probes > 1 ? (s2 - job->probes * m * m) / (job->probes - 1) : 0.0;
    }
    free(buf);
    return NULL;
}

int oracle_tree_estimate(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t mode, int32_t nthreads,
                         const int32_t *roots_in, int64_t n_roots, int32_t probes, uint64_t seed, double *mean,
                         double *var) {
    if (oracle_validate(n, row_ptr, col) || !roots_in || n_roots < 0 || probes < 1) return 1;
    if (mode != ORACLE_PIVOT_IP && mode != ORACLE_PIVOT_FULL) return 1;
    int32_t *rank = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *order = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *ap = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *adj = (int32_t *)malloc(((size_t)row_ptr[n] + 1) * sizeof(int32_t));
    int32_t *roots = (int32_t *)malloc(((size_t)n_roots + 1) * sizeof(int32_t));
    int rc = 0;
    if (!rank || !order || !ap || !adj || !roots) { rc = 2; goto done; }
    if (oracle_peel(n, row_ptr, col, NULL, rank, order) < 0) { rc = 2; goto done; }
    int32_t max_deg = 0;
    ap[0] = 0;
    for (int32_t r = 0; r < n; r++) {
        int32_t v = order[r], d = row_ptr[v + 1] - row_ptr[v];
        if (d > max_deg) max_deg = d;
        ap[r + 1] = ap[r] + d;
        int32_t *out = adj + ap[r];
        for (int32_t j = 0; j < d; j++) out[j] = rank[col[row_ptr[v] + j]];
        qsort(out, (size_t)d, sizeof(int32_t), cmp_int32);
    }
    for (int64_t i = 0; i < n_roots; i++) {
        if (roots_in[i] < 0 || roots_in[i] >= n) { rc = 1; goto done; }
        roots[i] = rank[roots_in[i]];
    }
    {
        graph_t g = {ap, adj, order, mode, 0};
        est_job_t job;
        memset(&job, 0, sizeof(job));
        job.g = &g;
        job.roots = roots;
        job.n_roots = n_roots;
        job.probes = probes;
        job.max_deg = max_deg;
        job.seed = seed;
        job.mean = mean;
        job.var = var;
        atomic_init(&job.next, 0);
        atomic_init(&job.failed, 0);
        int32_t nt = nthreads > 0 ? nthreads : oracle_default_threads();
        if (nt > 1024) nt = 1024;
        pthread_t th[1024];
        int32_t started = 0;
        for (int32_t t = 0; t < nt; t++) {
            if (pthread_create(&th[t], NULL, est_worker, &job) != 0) break;
            started++;
        }
        if (started == 0) est_worker(&job);
        for (int32_t t = 0; t < started; t++) pthread_join(th[t], NULL);
        if (atomic_load(&job.failed)) rc = 2;
    }
done:
    free(rank); free(order); free(ap); free(adj); free(roots);
    return rc;
}
