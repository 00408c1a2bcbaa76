/*
 * roargraph.h -- C ABI of the GB300 RoarGraph search library.
 *
 * RoarGraph (PVLDB 17(11), 2024) answers top-k maximum-inner-product queries
 * (Definition 1, Sec. 2.1.1) by beam search over a graph index built from a
 * query-base bipartite graph (Sec. 4.2). This library runs that search on the
 * GPU, plus the dense step of the index build.
 *
 * Conventions shared by every call:
 *  - All vectors are row-major FP32 unless stated; d must be a multiple of 4
 *    (rows start on 16-byte boundaries) and at most 1024.
 *  - delta(q, x) = -<q, x> (Sec. 5.1, MIPS); smaller is closer. Results are
 *    ordered by (distance ascending, id ascending).
 *  - Pointers marked "device" are CUDA device (or managed) memory; they are
 *    borrowed, never freed by the library, and must outlive every call that
 *    uses them (for an index: until roar_index_destroy returns).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls that
 *    take a stream only enqueue work; the return code reports argument
 *    validation and launch errors. Per-query outcomes go to `qstatus`.
 *  - No call aborts, throws or traps. Errors return a roar_status; the text of
 *    the last CUDA error is available from roar_last_error().
 */
#ifndef ROARGRAPH_H
#define ROARGRAPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ROAR_OK = 0,
    ROAR_EINVAL = 1,    /* bad argument (checked before any launch) */
    ROAR_ENOMEM = 2,    /* device or host allocation failed */
    ROAR_ECUDA = 3,     /* a CUDA call failed; see roar_last_error() */
    ROAR_EOVERFLOW = 4, /* per query: the visit cap ended the search early */
    ROAR_ETIMEOUT = 5,  /* a bounded wait gave up */
    ROAR_EBUSY = 6      /* resource in use (e.g. a server slot table is full) */
} roar_status;

typedef enum {
    ROAR_F32 = 0,       /* traversal on the FP32 rows themselves */
    ROAR_BF16 = 1,      /* traversal on a BF16 copy, FP32 re-rank */
    ROAR_FP8_E4M3 = 2   /* traversal on an FP8-E4M3 copy with per-row scales, FP32 re-rank */
} roar_dtype;

#define ROAR_NONE_ID 0xFFFFFFFFu   /* adjacency padding and unfilled result slots */
#define ROAR_MAX_RMAX 128          /* largest adjacency row width */
#define ROAR_MAX_L 1024            /* largest beam width (pool capacity) */
#define ROAR_MAX_K ROAR_MAX_L

typedef struct roar_index roar_index;
typedef struct roar_plan roar_plan;
typedef struct roar_server roar_server;

/* Serving-loop configuration (roar_server_create). */
typedef struct {
    int32_t ring_capacity;  /* query slots that may be in flight; 0: from memory_budget */
    int64_t memory_budget;  /* bytes of in-flight requests (see roar_server_create); 0: no byte limit */
    int32_t k_max;          /* largest k of a request */
    int32_t L_max;          /* largest L of a request (sizes each team's pool) */
    int32_t team_warps;     /* warps per query team, 0: the handle's tuning for L_max */
    int32_t idle_ms;        /* the kernel exits after this long without work (0: 50 ms) */
} roar_server_cfg;

/* Text for a status code (static storage). */
const char *roar_status_string(roar_status s);

/* Text of the last CUDA error seen by this thread (static storage, "" if none). */
const char *roar_last_error(void);

/*
 * Create a search handle over a resident index (Sec. 4.3: "the medoid of the
 * base data as the initial node").
 *   n, d          base rows and dimension (1 <= n < 2^31, d % 4 == 0, d <= 1024).
 *   base_f32      device [n][d] FP32 base vectors X. Required: the FP32 search
 *                 traverses it, the reduced-precision forms re-rank with it.
 *   trav_dtype    which copy the traversal reads (roar_dtype).
 *   base_trav     device [n][d] BF16 (uint16) or FP8-E4M3 (uint8) copy; NULL
 *                 for ROAR_F32. Produce it with roar_quantize.
 *   scales        device [n] FP32 per-row scales for ROAR_FP8_E4M3, else NULL.
 *   adj           device [n][rmax] uint32 out-neighbour ids, each row padded at
 *                 its end with ROAR_NONE_ID (the RoarGraph index of Alg. 1).
 *   rmax          row width, 1..ROAR_MAX_RMAX.
 *   entry         entry node id (< n), normally the medoid.
 *   max_visits    per-query cap on distinct visited nodes (0 = 16384, max 2^24);
 *                 sizes the library's scratch (see below).
 *   out           receives the handle.
 * Scratch: a 4-byte work counter at creation; on the first search that needs
 * them, per resident warp a visited bitmap of ceil(n/32) words and a log of
 * max_visits + ROAR_MAX_RMAX ids (growing them synchronises the device, so
 * run one search before capturing searches in a CUDA graph).
 * Searches on one handle must not overlap in time (enqueue them on one
 * stream); create one handle per concurrent stream.
 * Errors: ROAR_EINVAL, ROAR_ENOMEM, ROAR_ECUDA.
 */
roar_status roar_index_create(int64_t n, int32_t d, const float *base_f32, roar_dtype trav_dtype,
                              const void *base_trav, const float *scales, const uint32_t *adj,
                              int32_t rmax, uint32_t entry, uint32_t max_visits, roar_index **out);

/*
 * RoarGraph construction in the literal order of Alg. 1 (Sec. 4.2), composed
 * of the library's GPU parts, for checking them against the paper's steps on
 * small inputs (roar_build_index is the batched, fast form; see DESIGN):
 * training-query kNN (roar_knn, GPU); bipartite step; projection (Alg. 2)
 * with pivots in ascending id and every reverse edge applied before the next
 * pivot (host); connectivity enhancement with every base row searched over
 * the fixed G_pj (roar_search, GPU, width L_build) and its list pruned with
 * Alg. 3 without fill (roar_acquire, GPU), then the lists and reverse edges
 * applied in ascending row order (host); the final union; and the repair
 * (each unreachable node, smallest id first, gets an edge from its nearest
 * reachable node with a free slot, else the nearest gives up its last edge).
 * Every decision uses the search's fixed-order FP32 distance, ties by id.
 *   Arguments as roar_build_index (no thread count: the sequential steps run
 *   on one host thread; n <= 2^24, d % 8 == 0, d <= 512).
 *   stats [16]: [0] seconds, [6] pivots, [7] G_pj edges, [8] final edges,
 *   [9] nodes unreachable before the repair, [10] repairs.
 * Synchronises `stream`. Errors: ROAR_EINVAL, ROAR_ENOMEM, ROAR_ECUDA.
 */
roar_status roar_build_index_literal(const float *X_dev, int64_t n, int32_t d, const float *T_dev, int64_t nt,
                                     int32_t nq_depth, int32_t M, int32_t L_build, uint32_t *adj_dev,
                                     uint32_t *pj_dev, uint32_t *entry_out, double *stats, void *stream);

/*
 * The query-base bipartite graph G_bi of Alg. 1 (Sec. 4.2.2) from the
 * training queries' kNN lists: query node t has out-edges to its N_q - 1
 * nearest base rows after the first (N_out(t)); the nearest, x, gets the
 * out-edge x -> t. Every such edge is kept (no degree bound on B(x)).
 *   knn    device [nt][nqd] uint32, each row the training query's nqd nearest
 *          base ids in rank order (roar_knn), 2 <= nqd <= ROAR_MAX_RMAX + 1.
 *   off    device [n + 1] int64 out: B(x) = qids[off[x] .. off[x + 1]).
 *   qids   device [nt] uint32 out: query ids grouped by base node, ascending.
 *   nout   device [nt][nqd - 1] uint32 out: N_out(t) (knn without column 0).
 *   stats  host [2] out or NULL: base nodes with a query out-neighbour,
 *          largest |B(x)|.
 * Builds the CSR on the host (a counting sort of the nt rank-0 ids) and
 * synchronises `stream`. Errors: ROAR_EINVAL (also for an id >= n),
 * ROAR_ECUDA.
 */
roar_status roar_bipartite(const uint32_t *knn, int64_t nt, int32_t nqd, int64_t n, int64_t *off,
                           uint32_t *qids, uint32_t *nout, int64_t *stats, void *stream);

/*
 * A search handle over G_bi (roar_bipartite), for the ablation of Sec. 5.4:
 * roar_search on it runs the greedy search on the bipartite graph described
 * in Sec. 4.1, from a base node through its query out-neighbours to their
 * base out-neighbours. Only base nodes enter the pool and are scored (FP32,
 * the search's fixed order); expanding base node v scans N_out(t) for every
 * t in B(v), ascending, and the visit cap is checked before each such list.
 * Hops count expanded base nodes, visits count scored base nodes.
 *   n, d, base_f32, entry, max_visits   as roar_index_create (FP32 only).
 *   nout [nt][rn], bi_off [n + 1], bi_q [nt]   device arrays from roar_bipartite
 *                                              (rn = nqd - 1), borrowed.
 * The handle searches with one warp per query (roar_index_set_tuning with
 * more warps makes its searches fail with ROAR_EINVAL).
 * Errors: as roar_index_create.
 */
roar_status roar_index_create_bipartite(int64_t n, int32_t d, const float *base_f32, const uint32_t *nout,
                                        int32_t rn, int64_t nt, const int64_t *bi_off, const uint32_t *bi_q,
                                        uint32_t entry, uint32_t max_visits, roar_index **out);

/* Release a handle and its scratch (synchronises the device first). NULL is ignored. */
void roar_index_destroy(roar_index *idx);

/*
 * Tuning: shared-memory visited-table capacity 2^log2 slots per query
 * (5 <= log2 <= 15), 0 to choose from L automatically, or -1 for no shared
 * table. A query that visits more than half the table continues in its exact
 * global visited bitmap, so results never depend on this setting; speed and
 * occupancy do.
 * Errors: ROAR_EINVAL.
 */
roar_status roar_index_set_hash_log2(roar_index *idx, int32_t log2);

/*
 * Deletion by tombstones (Sec. 5.7): deleted rows still take part in routing
 * (they are visited and expanded like any other) but are left out of the
 * answers, which are the first k live entries of the final pool (after the
 * FP32 re-rank for the reduced-precision forms).
 *   bits  device bitmap of ceil(n/32) uint32 words, bit (id & 31) of word
 *         (id >> 5) set for a deleted row; NULL clears the tombstones. The
 *         caller owns it and may change its contents between searches; the
 *         handle keeps the pointer. Searches, uneven batches and servers
 *         created after this call read it; a captured plan keeps the pointer
 *         it was created with.
 * Errors: ROAR_EINVAL.
 */
roar_status roar_index_set_tombstones(roar_index *idx, const uint32_t *bits);

/*
 * Beam search (Sec. 4.3) of nq queries, each owned by one warp: start from
 * the entry, repeatedly expand the closest unexpanded pool entry, score its
 * unvisited out-neighbours, keep the first L under (distance, id), stop when
 * every pool entry is expanded. For ROAR_BF16 / ROAR_FP8_E4M3 handles the
 * traversal uses the reduced-precision copy, then every pool entry is
 * re-scored in FP32 and the first k of the re-sorted pool are returned.
 * FP32 distances use one fixed summation order (element i to lane
 * (i>>2)&31, fmaf per lane, then an xor butterfly 16,8,4,2,1), so results
 * are deterministic and independent of batch composition.
 *   queries   device [nq][d] FP32.
 *   k, L      1 <= k <= L <= ROAR_MAX_L.
 *   ids       device [nq][k] uint32 out; unfilled slots ROAR_NONE_ID.
 *   dist      device [nq][k] FP32 out (-<q,x>); unfilled slots +inf.
 *   visits    device [nq] uint32 out (distinct nodes scored), or NULL.
 *   hops      device [nq] uint32 out (expansions), or NULL.
 *   qstatus   device [nq] int32 out: ROAR_OK, ROAR_EOVERFLOW (visit cap hit;
 *             the pool so far is returned) or ROAR_EINVAL (the graph holds an
 *             id >= n, which is skipped); or NULL.
 * nq == 0 is a no-op. Errors: ROAR_EINVAL, ROAR_ECUDA.
 */
roar_status roar_search(roar_index *idx, const float *queries, int64_t nq, int32_t k, int32_t L,
                        uint32_t *ids, float *dist, uint32_t *visits, uint32_t *hops,
                        int32_t *qstatus, void *stream);

/*
 * roar_search with HOST buffers: copies the queries in, searches, copies the
 * results out and waits for completion before returning. Pinned host memory
 * gives the fastest copies. The device staging buffers are owned by the
 * handle and grow on demand. Same arguments and errors as roar_search.
 */
roar_status roar_search_host(roar_index *idx, const float *queries_host, int64_t nq, int32_t k,
                             int32_t L, uint32_t *ids_host, float *dist_host,
                             uint32_t *visits_host, uint32_t *hops_host, int32_t *qstatus_host,
                             void *stream);

/*
 * Uneven batch: roar_search with a per-query k and L (the paper's beam search,
 * Sec. 4.3, at each query's own beam width), all queries in one persistent
 * launch whose teams pull queries from a device work counter.
 *   k_dev, L_dev   device [nq] int32: 1 <= k <= L <= L_max per query; a query
 *                  outside that range gets qstatus ROAR_EINVAL and no output.
 *   out_off        device [nq] int64: first result slot of each query in
 *                  ids/dist (query q writes k[q] slots from out_off[q]).
 *   L_max          the largest L (sizes the shared-memory pool), <= ROAR_MAX_L.
 *   order          device [nq] int32 processing order (a permutation), or NULL
 *                  for 0..nq-1; results are the same in any order.
 * Other arguments as roar_search. Errors: ROAR_EINVAL, ROAR_ECUDA.
 */
roar_status roar_search_uneven(roar_index *idx, const float *queries, int64_t nq,
                               const int32_t *k_dev, const int32_t *L_dev, const int64_t *out_off,
                               int32_t L_max, const int32_t *order, uint32_t *ids, float *dist,
                               uint32_t *visits, uint32_t *hops, int32_t *qstatus, void *stream);

/*
 * Capture one roar_search_uneven launch (its buffers fixed) into a CUDA graph
 * for repeated replays with roar_plan_launch. With longest_first != 0 the
 * queries are processed in decreasing L (reads L_dev once, synchronising
 * `stream`), which shortens the launch's tail. The plan borrows every buffer
 * and the handle; the handle's scratch is sized before capture. Searches on
 * the handle must not overlap a replay. Errors: ROAR_EINVAL, ROAR_ENOMEM,
 * ROAR_ECUDA.
 */
roar_status roar_plan_create(roar_index *idx, const float *queries, int64_t nq, const int32_t *k_dev,
                             const int32_t *L_dev, const int64_t *out_off, int32_t L_max,
                             int32_t longest_first, uint32_t *ids, float *dist, uint32_t *visits,
                             uint32_t *hops, int32_t *qstatus, void *stream, roar_plan **out);

/* Replay a plan on `stream`. Errors: ROAR_EINVAL, ROAR_ECUDA. */
roar_status roar_plan_launch(roar_plan *plan, void *stream);

/* Release a plan (synchronises the device first). NULL is ignored. */
void roar_plan_destroy(roar_plan *plan);

/*
 * Launch tuning for the beam-width bucket that contains L (L <= 32, 64, 128,
 * 256, 512, 1024): team_warps in {1, 2, 4, 8} warps per query (32..256
 * threads), hash_log2 as in roar_index_set_hash_log2, blocks_per_sm_cap = 0
 * for the occupancy limit. Results never depend on the tuning.
 * Errors: ROAR_EINVAL.
 */
roar_status roar_index_set_tuning(roar_index *idx, int32_t L, int32_t team_warps, int32_t hash_log2,
                                  int32_t blocks_per_sm_cap);

/*
 * Autotune the bucket of L on a sample batch: times `repeats` searches of
 * each of 16 variants (team_warps {1,2,4,8} x visited-table mode {auto,
 * bitmap only, 2^10, 2^12}) and keeps the fastest in the handle.
 *   results  NULL or float[16] milliseconds per search, variant
 *            i = 4 * team_index + mode_index (1e30 where it cannot launch).
 *   best     NULL or the chosen variant index.
 * Allocates temporary outputs and synchronises `stream`.
 * Errors: ROAR_EINVAL, ROAR_ECUDA.
 */
roar_status roar_autotune(roar_index *idx, const float *queries, int64_t nq, int32_t k, int32_t L,
                          int32_t repeats, float *results, int32_t *best, void *stream);

/*
 * FP32 beam search that allocates nothing (no counterpart in the paper: it
 * serves callers that must not allocate device memory, such as code that runs
 * inside another framework's memory pool, which owns all device memory, or a
 * serving process that may not allocate, or synchronise through cudaMalloc,
 * once it is running). Same search and results as roar_search on an FP32
 * handle with the default tuning, but with no handle: the index is passed as
 * plain pointers (arguments as in roar_index_create and roar_search).
 * Scratch: one fixed 64 MiB device array inside the library (every GPU that
 * loads the library holds it until the process exits) holding a work counter
 * and, per resident warp, a visited bitmap of ceil(n/32) words and a visit
 * log of max_visits + ROAR_MAX_RMAX ids; the number of warps used is what fits
 * (fewer than roar_search on large n, so it can be slower). Sizes that do not
 * fit even 4 warps (4 * 4 * (ceil(n/32) + max_visits + 128) bytes above
 * 64 MiB - 512 bytes, e.g. n above about 133 million at the default
 * max_visits of 16384) return
 * ROAR_EINVAL with an explanation in roar_last_error().
 * The first call on each device, with that device current, looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture. Every call clears the parts that must start at zero,
 * but all calls share the one array: calls that overlap on the GPU (other
 * streams, other host threads) race and give wrong results.
 * Calls no cudaMalloc, cudaFree or other allocating routine.
 * Errors: ROAR_EINVAL, ROAR_ECUDA.
 */
roar_status roar_search_noalloc(int64_t n, int32_t d, const float *base_f32, const uint32_t *adj,
                                int32_t rmax, uint32_t entry, uint32_t max_visits,
                                const float *queries, int64_t nq, int32_t k, int32_t L,
                                uint32_t *ids, float *dist, uint32_t *visits, uint32_t *hops,
                                int32_t *qstatus, void *stream);

/*
 * Serving loop (continuous batching; no counterpart in the paper, whose
 * search runs one query at a time, Sec. 5.1). A server keeps the handle's
 * index resident and runs one persistent search kernel whose teams take
 * queries from a ring of slots in device memory as they are published, so
 * requests that arrive while others run start as soon as a team is free.
 * Queries, results and the publish / done marks move between host and device
 * by copies (pinned staging of the ring's size on the host), never through
 * host memory the kernel touches. Every query is the beam search of roar_search with its
 * request's k and L, bit-identical to searching it alone.
 * Admission, by memory: a query at (k, L) is charged
 *   4 d + 8 k + 24          its ring slot at its own k (query, results, counters)
 *   + 8 L                   its candidate pool
 *   + 4 * 2^ceil(log2(32 L)) the exact visited table for a beam of width L
 *                           (the kernel's sizing rule for its shared table)
 * bytes; a request of nq queries is charged nq times that. With
 * memory_budget > 0 a request is admitted only while the charges of the
 * requests in flight (submitted, not yet released by a poll) plus its own
 * stay within the budget; it is refused with ROAR_EBUSY otherwise and may be
 * retried after polls release requests (a request whose charge exceeds the
 * whole budget, or with more queries than ring slots, is ROAR_EINVAL). The
 * ring holds ring_capacity query slots of k_max results each (0: as many as
 * memory_budget / (4 d + 8 k_max + 24) allows, at most 2^26, or 65536 without
 * a budget); a request also needs free slots for all its queries.
 * The kernel's teams exit after idle_ms without work and the server
 * relaunches it when work is waiting; every wait in the kernel is bounded.
 * The server uses the handle's scratch: do not search the same handle while
 * a server runs on it. Errors: ROAR_EINVAL, ROAR_ENOMEM, ROAR_ECUDA.
 */
roar_status roar_server_create(roar_index *idx, const roar_server_cfg *cfg, roar_server **out);

/*
 * Submit nq queries (host [nq][d] FP32, copied) with one k and L. On success
 * *request_id identifies the request. ROAR_EBUSY: not enough free slots now.
 */
roar_status roar_server_submit(roar_server *srv, const float *q_host, int32_t nq, int32_t k, int32_t L,
                               uint64_t *request_id);

/*
 * Wait up to timeout_ms for a request. When complete: copies results to the
 * host arrays given (ids/dist [nq][k], visits/qstatus [nq]; any may be NULL),
 * writes the submit-to-completion latency in seconds, releases its slots and
 * returns ROAR_OK. ROAR_ETIMEOUT if not complete in time (poll again later);
 * ROAR_EINVAL for an unknown or already released request.
 */
roar_status roar_server_poll(roar_server *srv, uint64_t request_id, int32_t timeout_ms, uint32_t *ids,
                             float *dist, uint32_t *visits, int32_t *qstatus, double *latency_s);

/*
 * The ids of up to cap requests that are complete and not yet released
 * (oldest first) into ids (host [cap]); *n gets how many. A client polls
 * these instead of every request in flight. Errors: ROAR_EINVAL.
 */
roar_status roar_server_ready(roar_server *srv, uint64_t *ids, int32_t cap, int32_t *n);

/* out[10]: ring capacity, queries submitted, completed, released, kernel
 * launches, CTAs per launch, warps per team, kernel running (0/1), bytes
 * charged to requests in flight, memory budget. */
roar_status roar_server_stats(roar_server *srv, double *out);

/* Stop the kernel (bounded), join the poller and free the server. NULL is ignored. */
void roar_server_destroy(roar_server *srv);

/*
 * Reduced-precision copy of base rows for the traversal (a compression the
 * paper leaves open as orthogonal to the index, Sec. 4.3).
 *   X       device [n][d] FP32 (16-byte aligned, d % 4 == 0).
 *   dtype   ROAR_BF16: out is device [n][d] uint16 BF16 codes, round to
 *           nearest even; scales unused (may be NULL).
 *           ROAR_FP8_E4M3: out is device [n][d] uint8 codes with
 *           s_r = maxabs(row r) / 448 (IEEE division; 1 for an all-zero row)
 *           written to scales [n], code = E4M3(x / s_r) rounded to nearest
 *           even and saturated to +-448.
 * Asynchronous on `stream`. Errors: ROAR_EINVAL, ROAR_ECUDA.
 */
roar_status roar_quantize(const float *X, int64_t n, int32_t d, roar_dtype dtype, void *out,
                          float *scales, void *stream);

/*
 * Exact k-nearest neighbours under delta = -<t, x> (Definition 1, Sec. 2.1.1):
 * the preprocessing step of the construction ("ground truths" of the training
 * queries, Sec. 4.2.1) and the evaluation ground truth. Scores are computed
 * on the tensor cores (tcgen05, BF16 inputs, FP32 accumulation in TMEM) with
 * a fused running selection that keeps each row's 128 best candidates; these
 * are re-scored with exact FP32 dot products in the search's fixed order and
 * ids/dist get the first kk in (distance, id) order.
 *   T [nt][d], X [n][d]   device FP32, 16-byte aligned, d % 8 == 0, d <= 512.
 *   kk                    1..128, kk <= n.
 *   ids, dist             device [nt][kk] outputs.
 * Allocates and frees its own device scratch (BF16 copies of T and X with
 * rows padded to a multiple of 64 columns, and candidate buffers of 8 KB per
 * query row for up to 131,072 rows at a time)
 * and synchronises `stream` before returning. Errors: ROAR_EINVAL,
 * ROAR_ENOMEM, ROAR_ECUDA, ROAR_ETIMEOUT (a bounded tensor-core wait gave up).
 */
roar_status roar_knn(const float *T, int64_t nt, const float *X, int64_t n, int32_t d, int32_t kk,
                     uint32_t *ids, float *dist, void *stream);

/*
 * Testing hook of roar_knn's failure handling (no counterpart in the paper):
 * sets, for the whole process, the wall-time limit of each bounded wait
 * (mbarrier phase) inside the tensor-core kernel. ns < 0 restores the default
 * of 2 s. ns == 0 makes every wait give up as soon as its phase is found
 * incomplete, so a following roar_knn returns ROAR_ETIMEOUT through the same
 * path a real stall would take (the kernel waits for its copies and issued
 * MMAs, frees its TMEM and returns) without faulting anything. Affects
 * launches made after the call. Always returns ROAR_OK.
 */
roar_status roar_knn_set_wait_limit_ns(int64_t ns);

/*
 * Medoid entry point (Sec. 4.2.4, Sec. 4.3), read as the base row nearest in
 * FP64 L2 to the FP64 mean of the base rows, ties to the lower id.
 *   X_host  host [n][d] FP32. threads <= 0 uses every hardware thread.
 * Errors: ROAR_EINVAL.
 */
roar_status roar_medoid(const float *X_host, int64_t n, int32_t d, int32_t threads,
                        uint32_t *entry);

/*
 * AcquireNeighbors (Alg. 3, Sec. 4.2.3) for nx nodes at once, one warp each:
 * the candidates of node xs[i] are sorted by (delta(x, c), id) with
 * delta(x, c) = -dot(x, c) in the search's fixed FP32 summation order; the
 * first is kept, and each later candidate c is kept if delta(x, c) <
 * delta(c, r) for every kept r (same precision and order); at most M are kept,
 * and with fill the remaining budget is topped up from the other candidates in
 * sorted order. Candidates equal to x and ids already kept are skipped.
 *   X           device [n][d] FP32 rows, 16-byte aligned, d % 4 == 0, d <= 1024.
 *   xs          device [nx] uint32 node ids.
 *   cand        device [nx][cand_stride] uint32 candidate ids in any order;
 *               0xFFFFFFFF entries are padding; cand_stride <= 1024.
 *   ncand       device [nx] int32: entries of row i to read (clamped to
 *               [0, cand_stride]).
 *   M, fill     kept-list bound (1..64) and the fill flag.
 *   out         device [nx][M] uint32 out: the kept ids in order, padded with
 *               0xFFFFFFFF.
 *   out_cnt     device [nx] int32 out: ids kept, or -1 when xs[i] or one of
 *               its candidates is >= n (that row's out is all padding).
 *   sorted_out  device [nx][cand_stride] uint32 out or NULL: the valid
 *               candidates in the sorted order, padded with 0xFFFFFFFF.
 * Asynchronous on `stream`; the caller owns every buffer. Errors: ROAR_EINVAL
 * (sizes, pointers; checked before any launch), ROAR_ECUDA.
 */
roar_status roar_acquire(const float *X, int64_t n, int32_t d, const uint32_t *xs, int64_t nx,
                         const uint32_t *cand, int32_t cand_stride, const int32_t *ncand, int32_t M,
                         int32_t fill, uint32_t *out, int32_t *out_cnt, uint32_t *sorted_out,
                         void *stream);

/*
 * Build a RoarGraph index (Alg. 1): training-query kNN on the GPU (roar_knn,
 * depth nq_depth = N_q), bipartite graph, neighbourhood-aware projection with
 * AcquireNeighbors (Alg. 2, Alg. 3) on host threads, connectivity
 * enhancement with beam searches of width L_build and its AcquireNeighbors
 * pruning on the GPU (roar_search, roar_acquire), then reachability repair.
 * The rounds are batched (all pivots, then all reverse edges; enhancement in
 * chunks), deterministic for any thread count.
 *   X_dev [n][d], T_dev [nt][d]   device FP32 base rows and training queries.
 *   M                             out-degree bound of each phase; rows hold 2M.
 *   L_build                       candidate-set and beam size (M..ROAR_MAX_L).
 *   adj_dev                       device [n][2M] uint32 output, padded with
 *                                 ROAR_NONE_ID.
 *   pj_dev                        NULL or device [n][M] uint32 output: the
 *                                 projected graph G_pj before enhancement
 *                                 (for ablations), padded with ROAR_NONE_ID.
 *   entry_out                     the medoid.
 *   stats                         NULL or double[16]: total, kNN, projection,
 *                                 enhancement-search, reverse/merge and repair
 *                                 seconds; pivots; projected edges; final
 *                                 edges; unreachable before repair; repairs;
 *                                 unreachable after repair (0 unless every
 *                                 near candidate of a node is full).
 * Uses roughly n*(d*4 + 8*M) + nt*N_q*4 bytes of host memory and
 * synchronises `stream`. Errors: ROAR_EINVAL, ROAR_ENOMEM, ROAR_ECUDA.
 */
roar_status roar_build_index(const float *X_dev, int64_t n, int32_t d, const float *T_dev, int64_t nt,
                             int32_t nq_depth, int32_t M, int32_t L_build, int32_t threads,
                             uint32_t *adj_dev, uint32_t *pj_dev, uint32_t *entry_out, double *stats,
                             void *stream);

/*
 * Insertion through the saved bipartite graph (Sec. 5.7): rows n_old ..
 * n_total-1 of X_dev join the graph with the result of inserting them one at
 * a time, in id order. For row v: a beam search (width L, visit cap 16384) of
 * X[v]; the first pool entry that a training query is connected to (it is in
 * that query's N_out, or it is the query's pivot); q = the connected query
 * nearest to v; v's out-list = AcquireNeighbors with fill (Alg. 3, bound M)
 * over N_out(q), or over the search pool when no pool entry is connected;
 * each listed p gets p -> v, appended when p's row has room, else p's row and
 * v re-pruned to R with Alg. 3 (fill); v then joins N_out(q) while it has
 * room. All decisions use FP32 distances in the search's fixed summation
 * order.
 * The rows are processed in windows of `window` rows: their searches run in
 * one launch on the graph as it stands and record the nodes they expand (and
 * the pool's L-th distance at each); rows are then applied in order while the
 * search is still the one the sequential order runs: no node it expanded has
 * changed since, or those nodes only gained neighbours farther from the query
 * than that bound (which would not have entered the pool) without the visits
 * reaching the cap. The first row that fails is searched again in the next
 * window. So the result never depends on `window`; window = 1 is the plain
 * sequential order.
 *   X_dev        device [n_total][d] FP32 rows (the new rows already written).
 *   adj_dev      device [n_total][R] graph; rows >= n_old must be empty
 *                (ROAR_NONE_ID); updated in place. R <= 64, 1 <= M <= R.
 *   entry        search entry (< n_old).
 *   T_host       host [nt][d] FP32 training queries.
 *   pivot_host   host [nt]: each query's nearest base row.
 *   nout_host    host [nt][nout_cap] N_out lists, nout_cnt_host [nt] their
 *                lengths (nout_cap <= 1024); updated in place.
 *   window       rows per window, 1 .. 4096.
 *   chosen_q_host host [n_total - n_old] out: q per new row, or -1.
 *   stats        host [15] out or NULL: windows, searches run (rows searched
 *                more than once count each time), Alg. 3 lists computed,
 *                lists recomputed because N_out(q) grew, re-prune batches,
 *                rows re-pruned; then host seconds spent in setup (graph
 *                copy, connection lists, buffers), searches, lists, applying
 *                rows (re-prunes included), re-prunes, device graph updates
 *                and connected-query picks; then the windows whose apply
 *                stopped at a search that expanded a rewritten row, and
 *                those where every changed row it expanded was only appended
 *                to.
 * Synchronises `stream`. Uses about n_total * (R * 8 + 48) bytes of host
 * memory (the graph and, per entry, the insertion that appended it) plus the
 * connection lists, and a device copy of T_host. Errors: ROAR_EINVAL, ROAR_ENOMEM, ROAR_ECUDA.
 */
roar_status roar_insert(const float *X_dev, int64_t n_total, int32_t d, uint32_t *adj_dev, int32_t R,
                        uint32_t entry, int64_t n_old, const float *T_host, int64_t nt,
                        const uint32_t *pivot_host, uint32_t *nout_host, int32_t *nout_cnt_host,
                        int32_t nout_cap, int32_t M, int32_t L, int32_t window, int32_t *chosen_q_host,
                        double *stats, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ROARGRAPH_H */
