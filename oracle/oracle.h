/*
 * CPU oracle for maximal clique enumeration -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct restatement of what the GPU engine
 * computes. Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load it; the engine itself never links or calls it, and
 * this file shares no code, header, table or constant with the engine.
 *
 * What it computes (all exact integer work):
 *   M(G)   = the set of maximal cliques of a simple undirected graph G
 *            (Sec. II-A: a clique no vertex can be added to);
 *   count  = |M(G)|;
 *   hist[k]= number of maximal cliques with k vertices;
 *   hash   = sum over C in M(G) of h(C) mod 2^64, with
 *            h(C) = mix( sum_{c in C} mix(c + 1) + |C| * 0x9E3779B97F4A7C15 )
 *            on the INPUT vertex ids c, mix = the SplitMix64 output
 *            finaliser (Steele, Lea and Flood 2014). The paper only counts
 *            (Sec. IV-A); the histogram and this order-independent hash are
 *            this project's added outputs.
 *
 * How: the level-synchronous degeneracy peel (oracle_peel), then one
 * independent first-level subtree per vertex (Algorithm 3), each traversed
 * by Bron-Kerbosch with pivoting (Algorithm 2) or without (Algorithm 1).
 *
 * Status codes: 0 ok, 1 invalid graph, 2 out of memory, 5 histogram too short.
 */
#ifndef MCE_ORACLE_H
#define MCE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ORACLE_PIVOT_FULL = 0, /* Tomita: pivot from P u X (Sec. II-C) */
    ORACLE_PIVOT_IP = 1,   /* pivot from P u X_P only (Sec. III-E, partial induced subgraph) */
    ORACLE_NO_PIVOT = 2,   /* Algorithm 1 */
    /* flag, or-ed into a mode: one independent subtree per edge {v_i, v_j}
     * (Algorithm 4, Sec. III-B) instead of one per vertex (Algorithm 3) */
    ORACLE_SECOND_LEVEL = 8
};

/* 0 if (row_ptr, col) is a canonical simple undirected CSR over n vertices */
int oracle_validate(int32_t n, const int32_t *row_ptr, const int32_t *col);

/*
 * Degeneracy ordering by level-synchronous peeling (Sec. II-C, "Degeneracy
 * Ordering"; the GPU pre-processing of Sec. IV-A). Sub-round t removes, all
 * at once, S_t = { v remaining : deg_t(v) <= k_t } with
 * k_t = max(k_{t-1}, min remaining degree); vertices of S_t get consecutive
 * ranks in ascending input id; core[v] = k_t. Outputs are indexed by input
 * id except order[r] = the vertex of rank r. Any may be NULL.
 * Returns the number of sub-rounds (>= 0), or a negative status.
 */
int64_t oracle_peel(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t *core,
                    int32_t *rank, int32_t *order);

/*
 * All maximal cliques (Algorithm 3 over the peel order, Algorithm 2 or 1 per
 * subtree). hist[0..hist_len) is written (hist_len may be 0); *max_size gets
 * the largest clique size. Per-root arrays (indexed by input id of the root
 * vertex, each optional) receive that first-level subtree's clique count,
 * hash sum and number of recursive calls (tree nodes, root call included).
 * Roots are split across nthreads POSIX threads (<= 0: all online cores).
 * Returns 0, or 5 when hist_len <= *max_size (everything else still set).
 */
int oracle_mce(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t mode,
               int32_t nthreads, uint64_t *count, uint64_t *hash, uint64_t *hist,
               int32_t hist_len, int32_t *max_size, uint64_t *root_count,
               uint64_t *root_hash, uint64_t *root_nodes);

/*
 * Same as oracle_mce restricted to the first-level subtrees of the listed
 * root vertices (input ids); totals cover only those roots. Used to time a
 * bounded sample and to check sampled roots of very large graphs.
 */
int oracle_mce_roots(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t mode,
                     int32_t nthreads, const int32_t *roots, int64_t n_roots, uint64_t *count,
                     uint64_t *hash, uint64_t *hist, int32_t hist_len, int32_t *max_size,
                     uint64_t *root_count, uint64_t *root_hash, uint64_t *root_nodes);

/*
 * Per-root tree nodes and bitset word operations of the GPU formulation
 * (roots = NULL: all vertices). Word operations, with W = ceil(|P0|/32) for
 * the root's P0: at every call with P non-empty, W per pivot candidate
 * scanned (candidates in ascending rank, stopping at the first that reaches
 * the largest possible score), W for the branch set P - N(pivot), and 2W per
 * branch for the child's P and X_P. Used as the algorithmic work of the
 * integer-pipe roofline. Returns as oracle_mce (hist not collected).
 */
int oracle_mce_work(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t mode,
                    int32_t nthreads, const int32_t *roots, int64_t n_roots, uint64_t *root_nodes,
                    uint64_t *root_work);

/*
 * Per-root results of the listed roots (input ids) as oracle_mce_roots gives
 * them, except that a root whose subtree needs more than node_cap calls is
 * abandoned: its root_nodes entry is UINT64_MAX and its count and hash 0.
 * Lets a test pick roots the oracle can finish. Returns as oracle_mce_work.
 */
int oracle_mce_capped(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t mode, int32_t nthreads,
                      const int32_t *roots, int64_t n_roots, uint64_t node_cap, uint64_t *root_count,
                      uint64_t *root_hash, uint64_t *root_nodes);

/* count and hash of the maximal cliques of a complete multipartite graph with
 * `parts` parts of `part_size` consecutive ids starting at `first` (Moon-Moser
 * graphs have part_size 3): the transversals, enumerated directly. */
int oracle_multipartite(int32_t first, int32_t parts, int32_t part_size, uint64_t *count, uint64_t *hash);

/*
 * Knuth's unbiased estimate of each listed root's first-level subtree size
 * (Bron-Kerbosch calls, as oracle_mce_work's root_nodes) under pivot rule
 * `mode` (ORACLE_PIVOT_IP or ORACLE_PIVOT_FULL): mean[i] and sample variance
 * var[i] of `probes` random root-to-leaf paths of roots[i] (input ids), each
 * root's paths seeded from `seed` and its id. Returns 0, 1 (bad input) or 2.
 */
int oracle_tree_estimate(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t mode, int32_t nthreads,
                         const int32_t *roots, int64_t n_roots, int32_t probes, uint64_t seed, double *mean,
                         double *var);

/* h(C) for a clique given by input ids (any order) */
uint64_t oracle_clique_hash(const int32_t *ids, int32_t k);

/* number of threads oracle_mce would use for nthreads <= 0 */
int32_t oracle_default_threads(void);

#ifdef __cplusplus
}
#endif
#endif
