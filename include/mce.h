/*
 * mce.h -- C ABI of the GB300 (sm_103a) maximal clique enumeration engine.
 *
 * The engine enumerates every maximal clique of a simple undirected graph by
 * Bron-Kerbosch with pivoting (Algorithm 2 of "Parallelizing Maximal Clique
 * Enumeration on GPUs", Sec. II-B), over one independent first-level subtree
 * per vertex (Algorithm 3, Sec. II-C) in degeneracy order (Sec. II-C), with
 * each subtree walked depth-first on the GPU over bitset-encoded induced
 * subgraphs (Sec. III-A, III-D), a compact excluded set (Sec. III-E) and a
 * worker list for dynamic load balancing (Sec. III-C).
 *
 * Results are exact integers: the number of maximal cliques, the clique-size
 * histogram, and an order-independent 64-bit hash of the cliques,
 *     hash = sum over maximal cliques C of h(C)  (mod 2^64),
 *     h(C) = mix( sum_{c in C} mix(c + 1) + |C| * 0x9E3779B97F4A7C15 ),
 * with c the INPUT vertex ids and mix the SplitMix64 output finaliser
 * (z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27; z *= 0x94D049BB133111EB;
 * z ^= z>>31). The paper reports counts only (Sec. IV-A); the histogram and
 * the hash are added so that results can be compared exactly.
 *
 * Conventions shared by every entry point:
 *   - Return value: an MCE_* status. On failure nothing is written to the
 *     outputs unless stated; mce_last_error() gives a message.
 *   - Graphs are CSR with int32 ids and offsets: row_ptr[n+1], col[row_ptr[n]],
 *     each row sorted ascending, symmetric, no self-loops, no duplicates.
 *     Input that breaks any of these is rejected with MCE_EINVAL.
 *   - Ownership: the engine copies what it needs; caller buffers are never
 *     retained after a call returns.
 *   - Streams: all GPU work of a handle runs on the stream given at create
 *     time. NULL = a stream the handle creates, a blocking one, so that its
 *     work is ordered with work on the legacy default stream (where, for
 *     instance, an allocator passed below may hand out memory that the
 *     caller's pending kernels still use). Every call is synchronous with
 *     respect to the host on return, and mce_destroy waits for the handle's
 *     stream before it returns any memory to the allocator.
 *   - Threading: one handle must not be used by two host threads at once;
 *     distinct handles are independent.
 */
#ifndef MCE_H
#define MCE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define MCE_OK 0
#define MCE_EINVAL 1       /* bad argument or non-canonical graph */
#define MCE_ENOMEM 2       /* device or host allocation failed */
#define MCE_ECUDA 3        /* a CUDA call failed (message has the CUDA error) */
#define MCE_ETIMEOUT 4     /* a device wait saw no progress for opts.timeout_ms; results discarded */
#define MCE_ERANGE 5       /* hist_len <= max clique size; out->max_size is still set */
#define MCE_EUNSUPPORTED 6 /* graph beyond the engine's limits (degeneracy > MCE_MAX_DEGENERACY) */
#define MCE_EBUDGET 7      /* the run exceeded opts.run_budget_ms; results discarded */

/* largest degeneracy (= largest per-root candidate set |P|) the engine handles */
#define MCE_MAX_DEGENERACY 4096

/* create flags */
#define MCE_FLAG_DEVICE_PTRS 1u /* row_ptr/col (and graph_ptr) are device pointers */

/* pivot selection (Sec. III-D, III-E, IV-E) */
#define MCE_PIVOT_AUTO 0 /* IP when max_degree/degeneracy > 200, else IPX (Sec. IV-E heuristic) */
#define MCE_PIVOT_IP 1   /* pivot from P u X_P (partial induced subgraph) */
#define MCE_PIVOT_IPX 2  /* pivot from P u X_P u X_X (full induced subgraph) */

/* donation policy: a busy group may hand the child it is about to enter to an
 * idle group when the child's |P| >= donate_min_p and ... */
#define MCE_DONATE_PAPER 0 /* ... branches remain at this level AND at a shallower one (Sec. III-C) */
#define MCE_DONATE_EITHER 1 /* ... branches remain at this level OR at a shallower one */
#define MCE_DONATE_ANY 2   /* ... always (the donor may become idle right after) */

/* root ordering */
#define MCE_ORDER_PLAIN 0   /* roots by descending degeneracy rank within each width class */
#define MCE_ORDER_PRIORITY 1/* roots by descending opts.root_priority (e.g. learned work estimate);
                              roots whose priority is negative or NaN follow in the plain order */

typedef struct mce_graph mce_graph; /* opaque; owns its device copies */

/*
 * Optional device allocator. When given, every device allocation of the
 * handle goes through it (e.g. the PyTorch caching allocator); otherwise the
 * engine uses cudaMallocAsync/cudaFreeAsync on the handle's stream.
 * alloc returns NULL on failure (the call then fails with MCE_ENOMEM).
 */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *ctx;
} mce_allocator;

typedef struct {
    int32_t struct_size;   /* sizeof(mce_opts); set by mce_default_opts */
    int32_t pivot;         /* MCE_PIVOT_* */
    int32_t order;         /* MCE_ORDER_* */
    int32_t worker_list;   /* 1 = idle workers receive donated subtrees (Sec. III-C), 0 = off */
    int32_t donate_min_p;  /* donate a child only if its |P| >= this (Sec. III-C uses 10); 0 = automatic:
                            max(10, largest |P0| of the width class / 10) */
    int32_t blocks;        /* persistent blocks per width class; 0 = all that fit on the GPU */
    int32_t donate_policy; /* which busy groups may donate a child (Sec. III-C): MCE_DONATE_* */
    int32_t stats;         /* 1 = collect per-phase SM cycle counters (see mce_stats); slows the run.
                              Counting runs only: mce_run_list and subtree_level = 2 collect none */
    int64_t timeout_ms;    /* bound of every device-side wait (default 60000): an idle worker gives up
                              when no donation, no end of the launch and no heartbeat of a busy
                              worker has come for this long; work itself is never timed */
    /* optional DEVICE buffers, indexed by input vertex id, length n: the
     * clique count, hash sum and Bron-Kerbosch call count (tree nodes, root
     * call included) of each vertex's first-level subtree. */
    uint64_t *root_count;
    uint64_t *root_hash;
    uint64_t *root_nodes;
    /* DEVICE float[n] by input vertex id; read when order == MCE_ORDER_PRIORITY */
    const float *root_priority;
    /* optional DEVICE int32[n_roots] of distinct input vertex ids: only these
     * vertices' first-level subtrees (Algorithm 3) are enumerated, and every
     * result (count, hash, histogram, per-root arrays) covers only them.
     * NULL = all vertices. An id outside [0, n) fails with MCE_EINVAL. */
    const int32_t *roots;
    int64_t n_roots;
    int32_t tuned;         /* 1 = use the per-width-class settings mce_autotune chose for this handle */
    int32_t subtree_level; /* independent subtrees per vertex (0 or 1, Algorithm 3) or per edge
                            (2, Algorithm 4: R = {v_i, v_j}, no pivot step at the vertex level);
                            results are the same, tree nodes differ; opts.roots then selects
                            the edges of those vertices */
    int64_t run_budget_ms; /* the traversal stops once this much time has passed since its first
                              launch and the run fails with MCE_EBUDGET (default 600000, a safety
                              net that no run of the bundled workloads comes near); 0 = none */
    int32_t merge_wp;      /* one-warp width classes with rows of at most this many words share one
                              launch at the widest of them: 12 (default when 0), 4 or 1 (none) */
    int32_t block_warps;   /* warps per block of every traversal launch: 24 (default when 0), 16, 8
                              or 4 (never fewer than a group's warps) */
} mce_opts;

typedef struct {
    uint64_t count;       /* number of maximal cliques */
    uint64_t hash;        /* sum of h(C) mod 2^64 */
    int32_t max_size;     /* size of the largest maximal clique (0 for an empty graph) */
    int32_t degeneracy;   /* d: largest core number */
    uint64_t tree_nodes;  /* Bron-Kerbosch calls made (all subtrees) */
    uint64_t donations;   /* subtrees handed to idle workers */
    double ms_prep;       /* device time: validation + peel + orientation */
    double ms_traverse;   /* device time: all traversal launches */
} mce_result;

/* Fill *opts with defaults (IP/IPX auto, plain order, worker list on,
 * donate_min_p 0 = automatic, donate_policy MCE_DONATE_EITHER, timeout 60 s,
 * run budget 10 min). */
void mce_default_opts(mce_opts *opts);

/*
 * Build a handle for one graph: copy the CSR to the device, validate it,
 * compute the degeneracy order and core numbers by level-synchronous peeling
 * (Sec. II-C; ties inside a peel round by ascending id), and orient each
 * vertex's neighbours into later (its root P, Algorithm 3) and earlier (its
 * root X) lists.
 *   row_ptr, col  CSR as described above (host, or device with MCE_FLAG_DEVICE_PTRS)
 *   n             number of vertices (>= 0); m = number of undirected edges
 *                 (row_ptr[n] must equal 2m)
 *   alloc         optional device allocator (NULL = cudaMallocAsync)
 *   stream        cudaStream_t for all of the handle's work (NULL = own stream)
 *   out           receives the handle; NULL on failure
 * Errors: MCE_EINVAL (bad CSR), MCE_ENOMEM, MCE_ECUDA, MCE_EUNSUPPORTED.
 */
int mce_create(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t m, uint32_t flags,
               const mce_allocator *alloc, void *stream, mce_graph **out);

/*
 * Batched handle: G graphs with disjoint vertex ranges, graph g owning ids
 * [graph_ptr[g], graph_ptr[g+1]) of one concatenated CSR (no edge may cross
 * two ranges). All graphs are peeled and traversed together in the same
 * persistent launches; results are kept per graph.
 */
int mce_batch_create(const int32_t *graph_ptr, int32_t G, const int32_t *row_ptr, const int32_t *col,
                     int32_t n_total, int64_t m_total, uint32_t flags, const mce_allocator *alloc,
                     void *stream, mce_graph **out);

/*
 * Enumerate the maximal cliques of a single-graph handle.
 *   opts      NULL = defaults
 *   out       receives count, hash, sizes and statistics
 *   hist      optional HOST uint64[hist_len]: hist[k] = number of maximal
 *             cliques with k vertices (hist[0] = 0)
 * Errors: MCE_ERANGE if hist_len <= out->max_size (out is still filled;
 * retry with a longer hist), MCE_ETIMEOUT, MCE_ECUDA, MCE_ENOMEM, MCE_EINVAL.
 */
int mce_run(mce_graph *g, const mce_opts *opts, mce_result *out, uint64_t *hist, int32_t hist_len);

/*
 * mce_run_list -- every maximal clique of a single-graph handle, listed.
 * The paper's kernels only count the cliques they find; this call also writes
 * each clique C to buf as one record [|C|, id_1, ..., id_|C|] of int32 words (input
 * vertex ids, in no particular order; records in no particular order).
 *   buf        device memory of cap_words int32 words, or NULL: then only
 *              the size is computed (cap_words ignored)
 *   *words     receives the number of words the complete list needs
 *   out        the same results as mce_run (count, hash, ...)
 * opts as for mce_run; opts.roots restricts the listing to those roots'
 * first-level subtrees, which partition M(G) (every clique is listed under
 * its earliest vertex in the degeneracy order), so a list too large for one
 * buffer is produced root subset by root subset. Returns MCE_ERANGE when buf
 * is given and *words > cap_words: the records that fit are written, the
 * others dropped.
 */
int mce_run_list(mce_graph *g, const mce_opts *opts, int32_t *buf, int64_t cap_words, int64_t *words,
                 mce_result *out);

/*
 * Batched run: per_graph[G] results and hist[G * hist_len] (row g is graph
 * g's histogram), both HOST buffers; hist may be NULL. `total`, when not
 * NULL, receives the sums over all graphs.
 */
int mce_run_batch(mce_graph *g, const mce_opts *opts, mce_result *per_graph, uint64_t *hist,
                  int32_t hist_len, mce_result *total);

/*
 * Autotuner, within about budget_ms of device time; results never change.
 * (1) Bitset width of the one-warp width classes (rows of at most 12 words):
 * their roots run in one launch at the widest row width present, or rows of
 * 1-4 words share one 4-word launch and 12-word rows run alone, or every
 * class runs alone at its own width; the fastest over all those roots is
 * kept. (2) Then launch by launch, a coordinate search from the defaults over
 * the donation threshold (max(10, |P0|max/10), max(10, |P0|max/20),
 * max(10, |P0|max/5)), the donation rule (EITHER, PAPER, ANY), the block size
 * (16, 8 or 4 warps) and the grid (all blocks that fit, or one per SM),
 * keeping each change that is faster. Runs with opts.tuned = 1 use the result.
 */
int mce_autotune(mce_graph *g, const mce_opts *base, double budget_ms);
/* The chosen settings: HOST arrays of 9 width classes (0 / -1 = default;
 * warps = warps per block) and *merge_wp = the widest row width (1, 4 or 12)
 * whose one-warp classes share a launch. Any pointer may be NULL. */
int mce_get_tuning(const mce_graph *g, int32_t *donate_min_p, int32_t *donate_policy, int32_t *blocks,
                   int32_t *warps, int32_t *merge_wp);

/*
 * Capture one complete run (every memset and kernel of mce_run / mce_run_batch
 * with these opts: roots of |P0| = 0, then each width class, heaviest first)
 * into a CUDA graph kept by the handle; mce_run_prepared replays it with one
 * graph launch and one read-back. The opts' device buffers (per-root outputs,
 * priorities, subsets) must stay valid while the capture is kept. A new
 * mce_prepare or mce_destroy releases it.
 */
int mce_prepare(mce_graph *g, const mce_opts *opts);
int mce_run_prepared(mce_graph *g, mce_result *per_graph, uint64_t *hist, int32_t hist_len,
                     mce_result *total);

/* Handle facts (host values): n, m, G, degeneracy, max degree. Any may be NULL. */
int mce_graph_info(const mce_graph *g, int32_t *n, int64_t *m, int32_t *G, int32_t *degeneracy,
                   int32_t *max_degree);

/*
 * Device arrays of the handle's pre-processing, copied to HOST buffers of
 * length n (any may be NULL): core[v] = core number, rank[v] = position in
 * the degeneracy order, out_degree[v] = |P| of v's root (later neighbours).
 */
int mce_get_order(const mce_graph *g, int32_t *core, int32_t *rank, int32_t *out_degree);

/* Launch facts and optional counters of the handle's last mce_run / mce_run_batch. */
#define MCE_STATS_MAX_CLASSES 16
#define MCE_STATS_PHASES 9
typedef struct {
    int32_t struct_size;                         /* sizeof(mce_stats), set by the caller */
    int32_t n_classes;                           /* width classes launched (entries below) */
    int32_t class_wp[MCE_STATS_MAX_CLASSES];     /* 32-bit words per bitset row; 0 = roots with |P| = 0 */
    int32_t class_roots[MCE_STATS_MAX_CLASSES];  /* roots in the class */
    int32_t class_rows[MCE_STATS_MAX_CLASSES];   /* largest |P| of a root in the class */
    int32_t class_blocks[MCE_STATS_MAX_CLASSES]; /* persistent blocks launched */
    int32_t class_groups[MCE_STATS_MAX_CLASSES]; /* cooperating groups (subtree workers) */
    int32_t class_group_warps[MCE_STATS_MAX_CLASSES];
    double class_ms[MCE_STATS_MAX_CLASSES];      /* device time of the launch (CUDA events) */
    uint64_t kernel_launches;                    /* kernels of the last create + run */
    int64_t peel_rounds;                         /* sub-rounds of the degeneracy peel */
    /* with opts.stats = 1: SM cycles and event counts summed over groups, per
     * phase: 0 induced subgraph + excluded rows (count: tasks), 1 pivot
     * (candidates scored), 2 branch + child sets (tree nodes), 3 leaf
     * maximality tests (excluded rows tested), 4 excluded-set partition
     * (rows moved), 5 worker-list donations (donations), 6 idle wait
     * (subtrees received), 7 reloading the parent level on backtrack
     * (backtracks), 8 entering a one-word (compact) subtree from a wider
     * node (excluded rows re-encoded) */
    uint64_t phase_cycles[MCE_STATS_PHASES];
    uint64_t phase_counts[MCE_STATS_PHASES];
    /* narrowest row width whose roots the launch ran: one launch takes the
     * roots of every width class of at most 12 words, widest first */
    int32_t class_wp_min[MCE_STATS_MAX_CLASSES];
    /* the handle's degeneracy peel by stage (full grid, narrow stage of 16 CTAs, one block):
     * device time (globaltimer, ms) and sub-rounds */
    double peel_stage_ms[3];
    int32_t peel_stage_rounds[3];
    /* 1 when the peel's narrow stage ran as one 16-CTA thread-block cluster,
     * 0 when it ran on 16 blocks of the full grid or was not reached */
    int32_t peel_cluster;
} mce_stats;

int mce_get_stats(const mce_graph *g, mce_stats *out);

/*
 * mce_peel_noalloc -- the degeneracy peel of mce_create (core numbers and
 * order), for callers that must not allocate device memory. The paper has no
 * counterpart; it is a deployment variant of the same kernel.
 *
 * Who needs it: code whose device memory is owned by someone else -- a
 * serving process whose memory pool reserves the whole GPU up front (a
 * cudaMalloc of its own would fail or fragment the pool), or a plug-in that
 * runs inside another framework and may only use the buffers it is handed.
 *
 * It allocates nothing: its scratch is one file-scope static device array of
 * (5 * MCE_NOALLOC_MAX_VERTICES + MCE_NOALLOC_MAX_VERTICES / 32 + 1184) 32-bit
 * words (about 21 MB), which every GPU that loads the library holds until the
 * process exits. Graphs with n > MCE_NOALLOC_MAX_VERTICES are rejected with
 * MCE_EUNSUPPORTED.
 *   row_ptr, col  DEVICE CSR (canonical, as for mce_create); n vertices, m edges
 *   core, rank    DEVICE int32[n], by input id: core number, position in the order
 *   order         DEVICE int32[n]: order[r] = the vertex of rank r
 *   stream        cudaStream_t of the current device (NULL = default stream);
 *                 a stream of another device fails with MCE_EINVAL
 * Each call looks up the array's device address (cudaGetSymbolAddress) for
 * the current device, clears the parts that must start at zero, runs the
 * validation and the peel on `stream`, and synchronises that stream three
 * times to read the status words back: the call is synchronous on return.
 * Every call on a device shares the same array, so calls that overlap on the
 * GPU (two streams, two threads) race and must be serialised by the caller.
 * Each grid-barrier wait of the peel gives up after 60 s (MCE_ETIMEOUT).
 * Results equal mce_create's order (mce_get_order). Errors: MCE_EINVAL,
 * MCE_EUNSUPPORTED, MCE_ETIMEOUT, MCE_ECUDA; message in mce_last_error().
 */
#define MCE_NOALLOC_MAX_VERTICES (1 << 20)
int mce_peel_noalloc(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t m, int32_t *core,
                     int32_t *rank, int32_t *order, void *stream);

/* ------------------------------------------- learned work estimator
 * Not in the paper: a small network predicts log2 of each root's subtree
 * size (Bron-Kerbosch calls) from 16 root features; the prediction is only
 * used to order roots (opts.order = MCE_ORDER_PRIORITY), so results never
 * change. Features (int32, saturating at INT32_MAX), for a root v with
 * P0 = later and X0 = earlier neighbours in the degeneracy order:
 *   0 deg(v)             1 core(v)             2 |P0|              3 |X0|
 *   4 e(P0) + e(P0,X0')  5 e(P0)               6 e(P0,X0')         7 floor(2^16 e(P0) / C(|P0|,2))
 *   8 sum of deg(u), u in N(v)                 9 max / 10 min over u in P0 of |N(u) n P0|
 *  11 #u in P0 adjacent to all other P0        12 max / 13 sum of core(u) over u in P0
 *  14 max over x in X0' of |N(x) n P0|         15 C(|P0|,2) - e(P0)
 * where X0' = the 256 smallest input ids of X0 (all of X0 when smaller), which
 * bounds the cost of a root with a very large X0.
 * The network input is log2(1 + feature), standardised with per-feature
 * mean/std stored in the model. Layers: 16 -> 64 (ReLU) -> 64 (ReLU) -> 1,
 * weights rounded to BF16 (nearest even) in every use, biases and all
 * accumulation in FP32. Training minimises the mean squared error with Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8) on FP32 master weights. */
#define MCE_NUM_FEATURES 16
#define MCE_MODEL_HIDDEN 64
/* parameter vector: W1[64][16] b1[64] W2[64][64] b2[64] W3[64] b3 mean[16] std[16] */
#define MCE_MODEL_PARAMS (64 * 16 + 64 + 64 * 64 + 64 + 64 + 1 + 16 + 16)

typedef struct mce_model mce_model;

/* Root features of a single-graph or batched handle into DEVICE buffers of
 * n * 16 elements indexed [input id][feature]: raw int32 values and/or
 * log2(1 + value) as float (either may be NULL). */
int mce_root_features(mce_graph *g, int32_t *raw, float *feat);

/* New model from a HOST parameter vector (MCE_MODEL_PARAMS floats, every std > 0). */
int mce_model_create(const float *params, const mce_allocator *alloc, void *stream, mce_model **out);
int mce_model_get_params(const mce_model *m, float *params);
/* DEVICE feat[n][16] (log2 features) -> DEVICE out[n] predicted log2 subtree size */
int mce_model_predict(mce_model *m, const float *feat, int64_t n, float *out);
/* Gradient of the batch's mean squared error with respect to every trained
 * parameter (standardisation entries get 0), HOST grad[MCE_MODEL_PARAMS];
 * *loss = the mean squared error. DEVICE feat[batch][16], label[batch]. */
int mce_model_gradient(mce_model *m, const float *feat, const float *label, int32_t batch, float *grad,
                       float *loss);
/* One Adam step on the batch; *loss (HOST, may be NULL) = its mean squared error before the step. */
int mce_model_train_step(mce_model *m, const float *feat, const float *label, int32_t batch, float lr,
                         float *loss);
void mce_model_destroy(mce_model *m);

/* The learned order's input in one call, on the handle's stream: features and
 * predictions for the roots with |P0| >= min_p only (the others are cheap and
 * get -1, the lowest priority), written to DEVICE priority[n] by input id,
 * ready for opts.root_priority with MCE_ORDER_PRIORITY. */
int mce_predict_priority(mce_graph *g, mce_model *m, int32_t min_p, float *priority);

/* Release the handle and all its device memory. NULL is a no-op. */
void mce_destroy(mce_graph *g);

/* Message for the last failing call on this thread (never NULL). */
const char *mce_last_error(void);

/*
 * Self-test of the engine's device-side waits (no counterpart in the paper:
 * it checks that every wait is bounded, without faulting the GPU). It runs
 * one of the waits on its own, on `stream`, with a bound of timeout_ms
 * (1..10000) and returns what the engine would report:
 *   which 0  the worker list's idle wait on a flag nothing sets, one worker
 *            counted as busy, no heartbeat          -> MCE_ETIMEOUT
 *   which 1  the peel's grid barrier, one block short -> MCE_ETIMEOUT
 *   which 2  the idle wait with a busy worker posting heartbeats for three
 *            bounds, then ending the launch          -> MCE_OK
 * Synchronous on return; the context stays usable in every case.
 */
int mce_selftest_waits(int32_t which, int64_t timeout_ms, void *stream);

/*
 * Microbenchmarks for the roofline's denominators (no counterpart in the
 * paper, which quotes utilisation only): the chip's rate for the traversal's
 * unit of work measured on its own, at full occupancy (4 blocks of 256
 * threads per SM), on `stream`, synchronous on return.
 *   which 0  bitset word-ops: AND + POPC + the add that accumulates it, over
 *            independent register pairs       -> *rate in word-ops per second
 *   which 1  three-input logic ops (LOP3)      -> *rate in ops per second
 *   which 2  L2 reads: 40 passes over a 64 MiB buffer with 128-bit loads that
 *            bypass L1                         -> *rate in bytes per second
 * *sm_mhz (may be NULL): the SM clock during the timed launch (SM cycles over
 * globaltimer); *ms (may be NULL): the launch's duration.
 */
int mce_microbench(int32_t which, double *rate, double *sm_mhz, double *ms, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MCE_H */
