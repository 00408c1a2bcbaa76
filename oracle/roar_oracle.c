/*
 * RoarGraph CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded restatement of what RoarGraph (PVLDB 17(11),
 * 2024) computes: index construction (Alg. 1, Alg. 2, Alg. 3, Sec. 4.2) and the
 * beam search used to query it (Sec. 4.3). It exists to check the CUDA library
 * and is called only by the tests, by the smoke check and by the benchmark's
 * CPU-baseline leg. It shares no code, header or table with the CUDA library,
 * and the library never calls it.
 *
 * Readings of points the paper leaves open (each is also exercised by a test):
 *   - distance: delta(q, x) = -<q, x> (inner product, Sec. 5.1). Vectors are
 *     unit-norm, so this ranks like cosine.
 *   - search distances are FP32 and computed by orc_dot_fixed, whose summation
 *     order is fixed: element i goes to lane (i >> 2) & 31 of 32 lanes, each
 *     lane accumulates its elements in increasing i with fmaf from +0.0f, then
 *     a butterfly s_l = s_l + s_(l xor o) for o = 16, 8, 4, 2, 1; lane 0 is
 *     the result. Construction distances are FP64 in index order.
 *   - every ordering is the total order (distance ascending, id ascending).
 *   - entry point: the medoid, read as the base row closest (FP64 L2) to the
 *     FP64 mean of the base set (Sec. 4.2.4, Sec. 4.3).
 *   - search terminates when every pool entry has been expanded (Sec. 4.3,
 *     beam search of Sec. 2.1.2); a visit cap ends it early with status 4.
 *   - Alg. 1: every query keeps its bipartite edge to its 1-NN; several
 *     queries may share one 1-NN base node.
 *   - Alg. 2: candidates are gathered per element and gathering stops when
 *     |C| reaches L; N'(x) replaces earlier reverse edges of x; a reverse
 *     edge is appended when the target list has room, else the target list
 *     is re-pruned with Alg. 3.
 *   - Alg. 3: "for all p in Res" with a strict "<"; fill is on during the
 *     projection and off during connectivity enhancement.
 *   - Alg. 1, enhancement loop: each base row is searched over the projected graph
 *     G_pj (fixed during the pass); results are pruned without fill into G';
 *     the final list is N_pj(x) followed by N'(x) minus N_pj(x) (<= 2M).
 *   - reachability repair (not in the paper's algorithm, which claims
 *     reachability): every node not reachable from the entry gets an edge
 *     from its nearest reachable node.
 *
 * Parity status (each pin is a test under tests/, with hand-derived golden
 * cases under tests/golden/): the distance, the quantisers, the FP32 search,
 * the quantised search with its FP32 re-rank, Alg. 3, the projection and
 * connectivity enhancement of Alg. 1-2, the reachability repair, deletion
 * and insertion are each pinned by a hand-traced case as well as by
 * invariants; no code or data from the authors exists to compare whole
 * graphs against.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NONE 0xFFFFFFFFu
#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_EOVERFLOW 4

/* ------------------------------------------------------------------------ */
/* Distances                                                                 */
/* ------------------------------------------------------------------------ */

/* <q, x> in FP32, in the fixed 32-lane order described in the header. */
float orc_dot_fixed(const float *q, const float *x, int32_t d) {
    float lane[32];
    for (int l = 0; l < 32; ++l) lane[l] = 0.0f;
    for (int32_t i = 0; i < d; ++i) {
        int l = (int)((i >> 2) & 31);
        lane[l] = fmaf(q[i], x[i], lane[l]);
    }
    for (int o = 16; o >= 1; o >>= 1) {
        float next[32];
        for (int l = 0; l < 32; ++l) next[l] = lane[l] + lane[l ^ o];
        for (int l = 0; l < 32; ++l) lane[l] = next[l];
    }
    return lane[0];
}

/* delta(a, b) = -<a, b> in FP64, summed in index order (construction). */
static double dist64(const float *a, const float *b, int32_t d) {
    double s = 0.0;
    for (int32_t i = 0; i < d; ++i) s += (double)a[i] * (double)b[i];
    return -s;
}

double orc_dist_f64(const float *a, const float *b, int32_t d) { return dist64(a, b, d); }

/* Construction distances: FP64 in index order (prec 0, the construction's
 * default here) or -dot_fixed, the search's fixed-order FP32 dot (prec 1),
 * the precision a GPU construction takes its decisions in; held in a double
 * either way (FP32 -> FP64 is exact, so the orders agree). */
static double cdist(int prec, const float *a, const float *b, int32_t d) {
    return prec ? -(double)orc_dot_fixed(a, b, d) : dist64(a, b, d);
}

static int less_f32(float da, uint32_t ia, float db, uint32_t ib) {
    return da < db || (da == db && ia < ib);
}

static int less_f64(double da, uint32_t ia, double db, uint32_t ib) {
    return da < db || (da == db && ia < ib);
}

/* ------------------------------------------------------------------------ */
/* Number formats (BF16 and FP8-E4M3), written from their definitions.       */
/* ------------------------------------------------------------------------ */

static uint32_t f32_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float bits_f32(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

/* FP32 -> BF16 (1 sign, 8 exponent, 7 mantissa bits), round to nearest even. */
uint16_t orc_f32_to_bf16(float f) {
    uint32_t u = f32_bits(f);
    if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu) != 0)
        return (uint16_t)((u >> 16) | 0x0040u);            /* quiet NaN */
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;                                      /* ties to even */
    return (uint16_t)(u >> 16);
}

float orc_bf16_to_f32(uint16_t h) { return bits_f32((uint32_t)h << 16); }

/* FP8-E4M3 ("fn" variant): 1 sign, 4 exponent (bias 7), 3 mantissa bits, no
 * infinities, S.1111.111 is NaN, largest finite 448 = 1.75 * 2^8, smallest
 * subnormal 2^-9. Decoding follows the definition. */
float orc_e4m3_to_f32(uint8_t b) {
    int s = (b >> 7) & 1, e = (b >> 3) & 15, m = b & 7;
    float v;
    if (e == 15 && m == 7) return NAN;
    if (e == 0) v = ldexpf((float)m, -9);                   /* m/8 * 2^(1-7) */
    else v = ldexpf(1.0f + (float)m / 8.0f, e - 7);
    return s ? -v : v;
}

/* The 127 non-negative finite E4M3 values, ascending (code c -> vals[c]). */
static void e4m3_table(double *vals) {
    for (int c = 0; c <= 0x7E; ++c) vals[c] = (double)orc_e4m3_to_f32((uint8_t)c);
}

/* FP32 -> E4M3, round to nearest (ties to the even code), saturating to
 * +-448, NaN -> NaN. Nearest is found by bisection over the value table. */
static uint8_t f32_to_e4m3_tab(float f, const double *vals) {
    if (isnan(f)) return 0x7F;
    uint8_t sign = signbit(f) ? 0x80 : 0x00;
    double a = fabs((double)f);
    if (a >= vals[0x7E]) return (uint8_t)(sign | 0x7E);
    int lo = 0, hi = 0x7E;                      /* vals[lo] <= a < vals[hi] */
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (vals[mid] <= a) lo = mid; else hi = mid;
    }
    double dlo = a - vals[lo], dhi = vals[hi] - a;   /* exact in FP64 */
    int c;
    if (dlo < dhi) c = lo;
    else if (dhi < dlo) c = hi;
    else c = (lo & 1) ? hi : lo;
    return (uint8_t)(sign | c);
}

uint8_t orc_f32_to_e4m3(float f) {
    double vals[127];
    e4m3_table(vals);
    return f32_to_e4m3_tab(f, vals);
}

void orc_f32_to_e4m3_n(const float *in, int64_t n, uint8_t *out) {
    double vals[127];
    e4m3_table(vals);
    for (int64_t i = 0; i < n; ++i) out[i] = f32_to_e4m3_tab(in[i], vals);
}

void orc_f32_to_bf16_n(const float *in, int64_t n, uint16_t *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = orc_f32_to_bf16(in[i]);
}

/* Per-row BF16 copy (scale 1). */
void orc_quant_bf16(const float *X, int64_t n, int32_t d, uint16_t *out) {
    for (int64_t i = 0; i < n * (int64_t)d; ++i) out[i] = orc_f32_to_bf16(X[i]);
}

/* Per-row FP8 copy: s = maxabs(row) / 448 (IEEE FP32 division), code_i =
 * E4M3(x_i / s); an all-zero row gets s = 1. */
void orc_quant_e4m3(const float *X, int64_t n, int32_t d, uint8_t *out, float *scales) {
    double vals[127];
    e4m3_table(vals);
    for (int64_t r = 0; r < n; ++r) {
        const float *x = X + r * d;
        float m = 0.0f;
        for (int32_t i = 0; i < d; ++i) {
            float a = fabsf(x[i]);
            if (a > m) m = a;
        }
        float s = (m == 0.0f) ? 1.0f : m / 448.0f;
        scales[r] = s;
        for (int32_t i = 0; i < d; ++i) out[r * d + i] = f32_to_e4m3_tab(x[i] / s, vals);
    }
}

/* ------------------------------------------------------------------------ */
/* Beam search (Sec. 4.3), FP32 fixed-order distances.                      */
/* ------------------------------------------------------------------------ */

typedef struct { float d; uint32_t id; int checked; } ent32;

/* Insert (dd, u) into the sorted pool of capacity L, keeping the first L
 * entries of the total order ("added ... if closer ... or if the queue is not
 * filled", Sec. 4.3). */
static void pool_insert32(ent32 *pool, int32_t *size, int32_t L, float dd, uint32_t u) {
    int32_t pos;
    if (*size == L) {
        if (!less_f32(dd, u, pool[L - 1].d, pool[L - 1].id)) return;
        pos = L - 1;
    } else {
        pos = *size;
    }
    while (pos > 0 && less_f32(dd, u, pool[pos - 1].d, pool[pos - 1].id)) {
        pool[pos] = pool[pos - 1];
        --pos;
    }
    pool[pos].d = dd;
    pool[pos].id = u;
    pool[pos].checked = 0;
    if (*size < L) ++*size;
}

/* Traversal distance of base row u: plain FP32 (dtype 0), BF16 (1) or
 * FP8-E4M3 with a per-row scale (2): -(s_u * dot_fixed(q, float(xhat_u))). */
static float trav_dist(int dtype, const void *Xt, const float *scales, int32_t d,
                       const float *q, uint32_t u, float *tmp) {
    if (dtype == 0) return -orc_dot_fixed(q, (const float *)Xt + (int64_t)u * d, d);
    if (dtype == 1) {
        const uint16_t *r = (const uint16_t *)Xt + (int64_t)u * d;
        for (int32_t i = 0; i < d; ++i) tmp[i] = orc_bf16_to_f32(r[i]);
        return -orc_dot_fixed(q, tmp, d);
    }
    const uint8_t *r = (const uint8_t *)Xt + (int64_t)u * d;
    for (int32_t i = 0; i < d; ++i) tmp[i] = orc_e4m3_to_f32(r[i]);
    float s = scales ? scales[u] : 1.0f;
    return -(s * orc_dot_fixed(q, tmp, d));
}

/*
 * One beam search. Writes the final pool (size <= L, sorted) to pool_out,
 * returns status; *visits = |visited set|, *hops = expansions. If trace is
 * not NULL it receives the expanded node ids in order (capacity trace_cap).
 */
static int search_one(int dtype, const void *Xt, const float *scales, int64_t n, int32_t d,
                      const uint32_t *adj, int32_t rmax, uint32_t entry, const float *q,
                      int32_t L, uint32_t max_visits, ent32 *pool, int32_t *pool_size,
                      uint32_t *visits, uint32_t *hops, uint32_t *trace, int64_t trace_cap,
                      unsigned char *visited, float *tmp) {
    int status = ORC_OK;
    int32_t size = 0;
    uint32_t nvis = 0, nhops = 0;
    memset(visited, 0, (size_t)n);

    visited[entry] = 1;
    nvis = 1;
    pool_insert32(pool, &size, L, trav_dist(dtype, Xt, scales, d, q, entry, tmp), entry);

    for (;;) {
        int32_t sel = -1;
        for (int32_t i = 0; i < size; ++i)
            if (!pool[i].checked) { sel = i; break; }
        if (sel < 0) break;                       /* nothing left to expand */
        if (nvis >= max_visits) { status = ORC_EOVERFLOW; break; }
        pool[sel].checked = 1;
        uint32_t v = pool[sel].id;
        if (trace && (int64_t)nhops < trace_cap) trace[nhops] = v;
        ++nhops;
        for (int32_t j = 0; j < rmax; ++j) {
            uint32_t u = adj[(int64_t)v * rmax + j];
            if (u == ORC_NONE) continue;
            if ((int64_t)u >= n) { status = ORC_EINVAL; continue; }
            if (visited[u]) continue;
            visited[u] = 1;
            ++nvis;
            pool_insert32(pool, &size, L, trav_dist(dtype, Xt, scales, d, q, u, tmp), u);
        }
    }
    *pool_size = size;
    *visits = nvis;
    *hops = nhops;
    return status;
}

static int check_graph_args(int64_t n, int32_t d, int32_t rmax, uint32_t entry, int32_t k, int32_t L) {
    if (n <= 0 || d <= 0 || rmax <= 0 || (int64_t)entry >= n || k <= 0 || L <= 0 || k > L)
        return ORC_EINVAL;
    return ORC_OK;
}

/*
 * Batch beam search. dtype 0: Xt is FP32 [n][d] and the result is the pool's
 * first k entries. dtype 1 / 2: Xt is the BF16 / FP8 copy (scales for FP8),
 * the traversal runs on it and the whole final pool is re-ranked with exact
 * FP32 distances against X32 before the first k are taken.
 * Unfilled result slots get id 0xFFFFFFFF and distance +inf.
 * Returns 0, or 1 for bad arguments, 2 when out of memory. Per-query status
 * (0, or 4 when the visit cap ended the search) goes to qstatus.
 */
/*
 * Tombstones (deletion, Sec. 5.7): `tomb` is NULL or a bitmap of n bits (bit
 * id & 31 of word id >> 5) marking deleted rows. Deleted rows are searched
 * through like any other (the traversal, visits and hops do not change) but
 * are left out of the answer: the result is the first k entries of the final
 * (re-ranked) pool whose ids are not deleted.
 */
int orc_beam_search_tomb(int32_t dtype, const void *Xt, const float *scales, const float *X32,
                         int64_t n, int32_t d, const uint32_t *adj, int32_t rmax, uint32_t entry,
                         const float *Q, int64_t nq, int32_t k, int32_t L, uint32_t max_visits,
                         const uint32_t *tomb, uint32_t *ids, float *dist, uint32_t *visits,
                         uint32_t *hops, int32_t *qstatus) {
    if (check_graph_args(n, d, rmax, entry, k, L) || nq < 0 || dtype < 0 || dtype > 2)
        return ORC_EINVAL;
    if (dtype != 0 && X32 == NULL) return ORC_EINVAL;
    ent32 *pool = (ent32 *)malloc(sizeof(ent32) * (size_t)L);
    unsigned char *visited = (unsigned char *)malloc((size_t)n);
    float *tmp = (float *)malloc(sizeof(float) * (size_t)d);
    if (!pool || !visited || !tmp) { free(pool); free(visited); free(tmp); return ORC_ENOMEM; }
    for (int64_t qi = 0; qi < nq; ++qi) {
        const float *q = Q + qi * d;
        int32_t size = 0;
        uint32_t nv = 0, nh = 0;
        int st = search_one(dtype, Xt, scales, n, d, adj, rmax, entry, q, L, max_visits, pool,
                            &size, &nv, &nh, NULL, 0, visited, tmp);
        if (dtype != 0) {
            /* FP32 re-rank of every pool entry, then the total order again. */
            for (int32_t i = 0; i < size; ++i)
                pool[i].d = -orc_dot_fixed(q, X32 + (int64_t)pool[i].id * d, d);
            for (int32_t i = 1; i < size; ++i) {
                ent32 e = pool[i];
                int32_t j = i;
                while (j > 0 && less_f32(e.d, e.id, pool[j - 1].d, pool[j - 1].id)) {
                    pool[j] = pool[j - 1];
                    --j;
                }
                pool[j] = e;
            }
        }
        int32_t r = 0;
        for (int32_t i = 0; i < size && r < k; ++i) {
            const uint32_t u = pool[i].id;
            if (tomb && ((tomb[u >> 5] >> (u & 31)) & 1u)) continue;   /* deleted: not an answer */
            ids[qi * k + r] = u;
            dist[qi * k + r] = pool[i].d;
            ++r;
        }
        for (; r < k; ++r) {
            ids[qi * k + r] = ORC_NONE;
            dist[qi * k + r] = INFINITY;
        }
        if (visits) visits[qi] = nv;
        if (hops) hops[qi] = nh;
        if (qstatus) qstatus[qi] = st;
    }
    free(pool);
    free(visited);
    free(tmp);
    return ORC_OK;
}

int orc_beam_search(int32_t dtype, const void *Xt, const float *scales, const float *X32,
                    int64_t n, int32_t d, const uint32_t *adj, int32_t rmax, uint32_t entry,
                    const float *Q, int64_t nq, int32_t k, int32_t L, uint32_t max_visits,
                    uint32_t *ids, float *dist, uint32_t *visits, uint32_t *hops,
                    int32_t *qstatus) {
    return orc_beam_search_tomb(dtype, Xt, scales, X32, n, d, adj, rmax, entry, Q, nq, k, L, max_visits,
                                NULL, ids, dist, visits, hops, qstatus);
}

/* Single FP32 query with its expansion order (for hand-traced tests). */
int orc_beam_search_trace(const float *X, int64_t n, int32_t d, const uint32_t *adj, int32_t rmax,
                          uint32_t entry, const float *q, int32_t L, uint32_t max_visits,
                          uint32_t *pool_ids, float *pool_dist, int32_t *pool_size,
                          uint32_t *trace, int64_t trace_cap, uint32_t *visits, uint32_t *hops) {
    if (check_graph_args(n, d, rmax, entry, 1, L)) return ORC_EINVAL;
    ent32 *pool = (ent32 *)malloc(sizeof(ent32) * (size_t)L);
    unsigned char *visited = (unsigned char *)malloc((size_t)n);
    float *tmp = (float *)malloc(sizeof(float) * (size_t)d);
    if (!pool || !visited || !tmp) { free(pool); free(visited); free(tmp); return ORC_ENOMEM; }
    int32_t size = 0;
    int st = search_one(0, X, NULL, n, d, adj, rmax, entry, q, L, max_visits, pool, &size, visits,
                        hops, trace, trace_cap, visited, tmp);
    for (int32_t i = 0; i < size; ++i) {
        pool_ids[i] = pool[i].id;
        pool_dist[i] = pool[i].d;
    }
    *pool_size = size;
    free(pool);
    free(visited);
    free(tmp);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Search on the query-base bipartite graph G_bi (Alg. 1 bipartite step,     */
/* searched as in Sec. 4.1 and the ablation of Sec. 5.4).                    */
/* ------------------------------------------------------------------------ */

/*
 * G_bi from the training queries' kNN lists knn [nt][nqd] (rank order):
 * query node t has out-edges to knn[t][1..nqd-1] (N_out(t), the edge to its
 * nearest base node removed), and that nearest base node x = knn[t][0] has
 * the out-edge x -> t. Every such edge is kept: B(x) lists all t with
 * knn[t][0] = x, in ascending t. Written as CSR: off [n+1], qids [nt].
 */
int orc_bipartite(const uint32_t *knn, int64_t nt, int32_t nqd, int64_t n, int64_t *off, uint32_t *qids) {
    if (nt < 0 || nqd < 1 || n < 1) return ORC_EINVAL;
    for (int64_t x = 0; x <= n; ++x) off[x] = 0;
    for (int64_t t = 0; t < nt; ++t) {
        if ((int64_t)knn[t * nqd] >= n) return ORC_EINVAL;
        ++off[knn[t * nqd] + 1];
    }
    for (int64_t x = 0; x < n; ++x) off[x + 1] += off[x];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!fill) return ORC_ENOMEM;
    for (int64_t x = 0; x < n; ++x) fill[x] = off[x];
    for (int64_t t = 0; t < nt; ++t) qids[fill[knn[t * nqd]]++] = (uint32_t)t;   /* ascending t */
    free(fill);
    return ORC_OK;
}

/*
 * Beam search on G_bi (FP32 fixed-order distances). A greedy search on the
 * bipartite graph goes from a base node to its query out-neighbours and on
 * to their base out-neighbours (Sec. 4.1), so only base nodes enter the pool
 * and are scored: expanding base node v scans, for each t in B(v) in
 * ascending order, N_out(t) in rank order, visiting and scoring every base
 * node not yet visited. The visit cap is checked before each query node's
 * list is scanned (visits >= max_visits stops the search with status 4).
 * Everything else (pool, order, termination, output) is the beam search of
 * search_one. Returns status; results as orc_beam_search with dtype 0.
 */
int orc_beam_search_bi(const float *X, int64_t n, int32_t d, const uint32_t *knn, int64_t nt, int32_t nqd,
                       uint32_t entry, const float *Q, int64_t nq, int32_t k, int32_t L, uint32_t max_visits,
                       uint32_t *ids, float *dist, uint32_t *visits, uint32_t *hops, int32_t *qstatus) {
    if (n < 1 || d < 1 || nqd < 2 || (int64_t)entry >= n || k < 1 || L < k || nq < 0) return ORC_EINVAL;
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    uint32_t *qids = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nt > 0 ? nt : 1));
    ent32 *pool = (ent32 *)malloc(sizeof(ent32) * (size_t)L);
    unsigned char *visited = (unsigned char *)malloc((size_t)n);
    int rc = ORC_ENOMEM;
    if (!off || !qids || !pool || !visited) goto done;
    rc = orc_bipartite(knn, nt, nqd, n, off, qids);
    if (rc != ORC_OK) goto done;
    for (int64_t qi = 0; qi < nq; ++qi) {
        const float *q = Q + qi * d;
        int st = ORC_OK;
        int32_t size = 0;
        uint32_t nvis = 1, nh = 0;
        memset(visited, 0, (size_t)n);
        visited[entry] = 1;
        pool_insert32(pool, &size, L, -orc_dot_fixed(q, X + (int64_t)entry * d, d), entry);
        for (;;) {
            int32_t sel = -1;
            for (int32_t i = 0; i < size; ++i)
                if (!pool[i].checked) { sel = i; break; }
            if (sel < 0) break;
            if (nvis >= max_visits) { st = ORC_EOVERFLOW; break; }
            pool[sel].checked = 1;
            const uint32_t v = pool[sel].id;
            ++nh;
            int stop = 0;
            for (int64_t j = off[v]; j < off[v + 1] && !stop; ++j) {
                if (nvis >= max_visits) { st = ORC_EOVERFLOW; stop = 1; break; }
                const uint32_t *nout = knn + (int64_t)qids[j] * nqd + 1;
                for (int32_t r = 0; r < nqd - 1; ++r) {
                    const uint32_t u = nout[r];
                    if (u == ORC_NONE) continue;
                    if ((int64_t)u >= n) { st = ORC_EINVAL; continue; }
                    if (visited[u]) continue;
                    visited[u] = 1;
                    ++nvis;
                    pool_insert32(pool, &size, L, -orc_dot_fixed(q, X + (int64_t)u * d, d), u);
                }
            }
            if (stop) break;
        }
        int32_t r = 0;
        for (; r < size && r < k; ++r) {
            ids[qi * k + r] = pool[r].id;
            dist[qi * k + r] = pool[r].d;
        }
        for (; r < k; ++r) {
            ids[qi * k + r] = ORC_NONE;
            dist[qi * k + r] = INFINITY;
        }
        if (visits) visits[qi] = nvis;
        if (hops) hops[qi] = nh;
        if (qstatus) qstatus[qi] = st;
    }
    rc = ORC_OK;
done:
    free(off);
    free(qids);
    free(pool);
    free(visited);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Exact kNN (Definition 1, Sec. 2.1.1) in FP64, ties to the lower id.       */
/* ------------------------------------------------------------------------ */

int orc_knn_f64(const float *Q, int64_t nq, const float *X, int64_t n, int32_t d, int32_t k,
                uint32_t *ids, double *dist) {
    if (nq < 0 || n <= 0 || d <= 0 || k <= 0 || k > n) return ORC_EINVAL;
    for (int64_t qi = 0; qi < nq; ++qi) {
        uint32_t *oi = ids + qi * k;
        double *od = dist + qi * k;
        int32_t size = 0;
        for (int64_t j = 0; j < n; ++j) {
            double dd = dist64(Q + qi * d, X + j * d, d);
            uint32_t u = (uint32_t)j;
            int32_t pos;
            if (size == k) {
                if (!less_f64(dd, u, od[k - 1], oi[k - 1])) continue;
                pos = k - 1;
            } else {
                pos = size++;
            }
            while (pos > 0 && less_f64(dd, u, od[pos - 1], oi[pos - 1])) {
                od[pos] = od[pos - 1];
                oi[pos] = oi[pos - 1];
                --pos;
            }
            od[pos] = dd;
            oi[pos] = u;
        }
    }
    return ORC_OK;
}

/* Medoid entry point (Sec. 4.2.4, Sec. 4.3): the base row nearest (FP64 L2)
 * to the FP64 mean of the base set, ties to the lower id. */
int64_t orc_medoid(const float *X, int64_t n, int32_t d) {
    if (n <= 0 || d <= 0) return -1;
    double *mu = (double *)calloc((size_t)d, sizeof(double));
    if (!mu) return -1;
    for (int64_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < d; ++j) mu[j] += (double)X[i * d + j];
    for (int32_t j = 0; j < d; ++j) mu[j] /= (double)n;
    int64_t best = 0;
    double bestd = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t j = 0; j < d; ++j) {
            double t = (double)X[i * d + j] - mu[j];
            s += t * t;
        }
        if (s < bestd) { bestd = s; best = i; }
    }
    free(mu);
    return best;
}

/* ------------------------------------------------------------------------ */
/* Construction (Alg. 1-3)                                                    */
/* ------------------------------------------------------------------------ */

typedef struct { uint32_t *v; int32_t n; int32_t cap; } ulist;

static int ul_push(ulist *l, uint32_t x) {
    if (l->n == l->cap) {
        int32_t nc = l->cap ? 2 * l->cap : 8;
        uint32_t *nv = (uint32_t *)realloc(l->v, sizeof(uint32_t) * (size_t)nc);
        if (!nv) return ORC_ENOMEM;
        l->v = nv;
        l->cap = nc;
    }
    l->v[l->n++] = x;
    return ORC_OK;
}

static int ul_has(const ulist *l, uint32_t x) {
    for (int32_t i = 0; i < l->n; ++i)
        if (l->v[i] == x) return 1;
    return 0;
}

static void ul_free_all(ulist *ls, int64_t n) {
    if (!ls) return;
    for (int64_t i = 0; i < n; ++i) free(ls[i].v);
    free(ls);
}

typedef struct { double d; uint32_t id; } ent64;

static int cmp_ent64(const void *a, const void *b) {
    const ent64 *x = (const ent64 *)a, *y = (const ent64 *)b;
    if (less_f64(x->d, x->id, y->d, y->id)) return -1;
    if (less_f64(y->d, y->id, x->d, x->id)) return 1;
    return 0;
}

/*
 * Alg. 3 AcquireNeighbors(x, C, M): C is sorted by (delta(x, c), id).
 * Res starts with the closest candidate; each later candidate c is added iff
 * delta(x, c) < delta(c, p) for every p already in Res; stop once |Res| = M.
 * With fill, the remaining candidates are appended in order until |Res| = M.
 * Returns |Res| written to res (capacity M).
 */
static int32_t acquire_neighbors(int prec, const float *X, int32_t d, uint32_t x, const ent64 *C, int32_t nc,
                                 int32_t M, int fill, uint32_t *res) {
    int32_t nr = 0;
    const float *xv = X + (int64_t)x * d;
    for (int32_t i = 0; i < nc && nr < M; ++i) {
        uint32_t c = C[i].id;
        if (c == x) continue;
        int dup = 0;
        for (int32_t j = 0; j < nr; ++j)
            if (res[j] == c) dup = 1;
        if (dup) continue;
        if (nr == 0) { res[nr++] = c; continue; }            /* the closest candidate */
        double dxc = cdist(prec, xv, X + (int64_t)c * d, d);
        int keep = 1;
        for (int32_t j = 0; j < nr && keep; ++j)
            if (!(dxc < cdist(prec, X + (int64_t)c * d, X + (int64_t)res[j] * d, d))) keep = 0;
        if (keep) res[nr++] = c;
    }
    if (fill) {
        for (int32_t i = 0; i < nc && nr < M; ++i) {
            uint32_t c = C[i].id;
            if (c == x) continue;
            int dup = 0;
            for (int32_t j = 0; j < nr; ++j)
                if (res[j] == c) dup = 1;
            if (!dup) res[nr++] = c;
        }
    }
    return nr;
}

/* Exported for tests: C given as ids already sorted by the caller's order;
 * distances delta(x, c) are recomputed here. */
int32_t orc_acquire_neighbors(const float *X, int64_t n, int32_t d, uint32_t x, const uint32_t *cand,
                              int32_t nc, int32_t M, int32_t fill, uint32_t *res) {
    if ((int64_t)x >= n || nc < 0 || M <= 0) return -1;
    ent64 *C = (ent64 *)malloc(sizeof(ent64) * (size_t)(nc > 0 ? nc : 1));
    if (!C) return -1;
    for (int32_t i = 0; i < nc; ++i) {
        if ((int64_t)cand[i] >= n) { free(C); return -1; }
        C[i].id = cand[i];
        C[i].d = dist64(X + (int64_t)x * d, X + (int64_t)cand[i] * d, d);
    }
    int32_t r = acquire_neighbors(0, X, d, x, C, nc, M, fill, res);
    free(C);
    return r;
}

/* Alg. 3 again, with every distance in FP32 by the search's fixed order:
 * delta(a, b) = -orc_dot_fixed(a, b). The paper fixes no precision for the
 * pruning test; this form takes each keep / drop decision in the precision a
 * GPU implementation takes it in (FP32, fixed summation order), so the two
 * can be compared id for id. C is given as ids in the caller's order. */
int32_t orc_acquire_neighbors_f32(const float *X, int64_t n, int32_t d, uint32_t x, const uint32_t *cand,
                                  int32_t nc, int32_t M, int32_t fill, uint32_t *res) {
    if ((int64_t)x >= n || nc < 0 || M <= 0) return -1;
    for (int32_t i = 0; i < nc; ++i)
        if ((int64_t)cand[i] >= n) return -1;
    const float *xv = X + (int64_t)x * d;
    int32_t nr = 0;
    for (int32_t i = 0; i < nc && nr < M; ++i) {
        const uint32_t c = cand[i];
        if (c == x) continue;
        int dup = 0;
        for (int32_t j = 0; j < nr; ++j)
            if (res[j] == c) dup = 1;
        if (dup) continue;
        if (nr == 0) { res[nr++] = c; continue; }            /* the closest candidate */
        const float *cv = X + (int64_t)c * d;
        const float dxc = -orc_dot_fixed(xv, cv, d);
        int keep = 1;
        for (int32_t j = 0; j < nr && keep; ++j)
            if (!(dxc < -orc_dot_fixed(cv, X + (int64_t)res[j] * d, d))) keep = 0;
        if (keep) res[nr++] = c;
    }
    if (fill) {
        for (int32_t i = 0; i < nc && nr < M; ++i) {
            const uint32_t c = cand[i];
            if (c == x) continue;
            int dup = 0;
            for (int32_t j = 0; j < nr; ++j)
                if (res[j] == c) dup = 1;
            if (!dup) res[nr++] = c;
        }
    }
    return nr;
}

/* Reverse-edge update of Alg. 2 and of Alg. 1's enhancement loop: give p the edge
 * p -> x. Skip when present; append when there is room; otherwise re-prune
 * N(p) U {x} with Alg. 3. */
static int reverse_update(int prec, const float *X, int32_t d, ulist *G, uint32_t p, uint32_t x, int32_t M,
                          int fill, ent64 *buf, uint32_t *res, int64_t *reprunes) {
    ulist *lp = &G[p];
    if (ul_has(lp, x)) return ORC_OK;
    if (lp->n < M) return ul_push(lp, x);
    const float *pv = X + (int64_t)p * d;
    int32_t nc = 0;
    for (int32_t i = 0; i < lp->n; ++i) {
        buf[nc].id = lp->v[i];
        buf[nc].d = cdist(prec, pv, X + (int64_t)lp->v[i] * d, d);
        ++nc;
    }
    buf[nc].id = x;
    buf[nc].d = cdist(prec, pv, X + (int64_t)x * d, d);
    ++nc;
    qsort(buf, (size_t)nc, sizeof(ent64), cmp_ent64);
    int32_t nr = acquire_neighbors(prec, X, d, p, buf, nc, M, fill, res);
    lp->n = 0;
    for (int32_t i = 0; i < nr; ++i)
        if (ul_push(lp, res[i])) return ORC_ENOMEM;
    ++*reprunes;
    return ORC_OK;
}

/* FP64 beam search over adjacency lists G (used by connectivity enhancement,
 * the enhancement loop of Alg. 1). Same algorithm as search_one with FP64 distances and no
 * visit cap. Writes the final pool (sorted, size returned). */
static int32_t beam_search_f64_lists(int prec, const float *X, int64_t n, int32_t d, const ulist *G,
                                     uint32_t entry, const float *q, int32_t L, ent64 *pool,
                                     unsigned char *checked, unsigned char *visited) {
    int32_t size = 0;
    memset(visited, 0, (size_t)n);
    visited[entry] = 1;
    pool[0].d = cdist(prec, q, X + (int64_t)entry * d, d);
    pool[0].id = entry;
    checked[0] = 0;
    size = 1;
    for (;;) {
        int32_t sel = -1;
        for (int32_t i = 0; i < size; ++i)
            if (!checked[i]) { sel = i; break; }
        if (sel < 0) break;
        checked[sel] = 1;
        uint32_t v = pool[sel].id;
        for (int32_t j = 0; j < G[v].n; ++j) {
            uint32_t u = G[v].v[j];
            if (visited[u]) continue;
            visited[u] = 1;
            double dd = cdist(prec, q, X + (int64_t)u * d, d);
            int32_t pos;
            if (size == L) {
                if (!less_f64(dd, u, pool[L - 1].d, pool[L - 1].id)) continue;
                pos = L - 1;
            } else {
                pos = size++;
            }
            while (pos > 0 && less_f64(dd, u, pool[pos - 1].d, pool[pos - 1].id)) {
                pool[pos] = pool[pos - 1];
                checked[pos] = checked[pos - 1];
                --pos;
            }
            pool[pos].d = dd;
            pool[pos].id = u;
            checked[pos] = 0;
        }
    }
    return size;
}

/*
 * Reachability repair (an addition: the paper states that connectivity
 * enhancement makes every base node reachable, Sec. 4.2.3, but its
 * algorithm does not guarantee it). adj [n][R]: rows of ids, each compact
 * (edges first, then 0xFFFFFFFF padding), modified in place. While some node
 * is not reachable from the entry:
 *   u = the smallest unreachable id;
 *   among the reachable nodes with a free slot, r = the nearest to u
 *     (FP64 delta(u, r) = -<x_u, x_r>, ties to the lower id): u is appended
 *     to r's row;
 *   when every reachable node is full, r = the nearest of them (same order)
 *     gives up its last edge, which becomes r -> u;
 *   reachability is recomputed (breadth-first from the entry).
 * Returns the number of repairs (-1 when out of memory); *unreachable0 gets
 * the number of nodes unreachable before the first repair.
 */
static int64_t repair_prec(int prec, const float *X, int64_t n, int32_t d, uint32_t *adj, int32_t R,
                           uint32_t entry, int64_t *unreachable0) {
    unsigned char *reach = (unsigned char *)malloc((size_t)n);
    uint32_t *queue = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    if (!reach || !queue) { free(reach); free(queue); return -1; }
    int64_t repairs = 0;
    for (;;) {
        /* breadth-first marking from the entry */
        memset(reach, 0, (size_t)n);
        int64_t head = 0, tail = 0;
        reach[entry] = 1;
        queue[tail++] = entry;
        while (head < tail) {
            const uint32_t v = queue[head++];
            for (int32_t j = 0; j < R; ++j) {
                const uint32_t w = adj[(int64_t)v * R + j];
                if (w == ORC_NONE || (int64_t)w >= n || reach[w]) continue;
                reach[w] = 1;
                queue[tail++] = w;
            }
        }
        if (repairs == 0 && unreachable0) *unreachable0 = n - tail;
        if (tail == n) break;
        uint32_t u = 0;
        while (reach[u]) ++u;
        int64_t best = -1, bestfull = -1;
        double bd = INFINITY, bdf = INFINITY;
        for (int64_t r = 0; r < n; ++r) {
            if (!reach[r]) continue;
            const double dd = cdist(prec, X + (int64_t)u * d, X + r * d, d);
            if (adj[r * R + R - 1] == ORC_NONE) {
                if (dd < bd) { bd = dd; best = r; }
            } else if (dd < bdf) {
                bdf = dd;
                bestfull = r;
            }
        }
        if (best >= 0) {
            int32_t j = 0;
            while (adj[best * R + j] != ORC_NONE) ++j;
            adj[best * R + j] = u;
        } else {
            adj[bestfull * R + R - 1] = u;
        }
        ++repairs;
    }
    free(reach);
    free(queue);
    return repairs;
}

int64_t orc_repair(const float *X, int64_t n, int32_t d, uint32_t *adj, int32_t R, uint32_t entry,
                   int64_t *unreachable0) {
    return repair_prec(0, X, n, d, adj, R, entry, unreachable0);
}

/*
 * Full construction (Alg. 1): bipartite graph from the training queries'
 * kNN lists, neighbourhood-aware projection (Alg. 2 with Alg. 3),
 * connectivity enhancement, then reachability repair.
 *
 *   X [n][d]: base vectors; nt: number of training queries.
 *   knn [nt][nqd]: each training query's nqd nearest base ids, rank order.
 *   M: out-degree bound; L: candidate-set / beam size.
 *   entry: the search entry (the medoid).
 *   pj_out [n][M]: the projected graph G_pj, padded with 0xFFFFFFFF (may be NULL).
 *   adj_out [n][2M]: the final index, padded with 0xFFFFFFFF.
 *   stats[8]: pivots, projection reprunes, CE reprunes, repairs,
 *             pj edges, final edges, isolated-in-G_pj, unreachable-before-repair.
 */
int orc_build_prec(const float *X, int64_t n, int64_t nt, int32_t d,
                   const uint32_t *knn, int32_t nqd, int32_t M, int32_t L, uint32_t entry,
                   uint32_t *pj_out, uint32_t *adj_out, int64_t *stats, int32_t prec) {
    if (n <= 0 || nt < 0 || d <= 0 || nqd < 1 || M <= 0 || L <= 0 || (int64_t)entry >= n)
        return ORC_EINVAL;
    int rc = ORC_ENOMEM;
    int64_t pivots = 0, proj_reprunes = 0, ce_reprunes = 0, repairs = 0;
    ulist *B = (ulist *)calloc((size_t)n, sizeof(ulist));   /* base -> training query */
    ulist *Gpj = (ulist *)calloc((size_t)n, sizeof(ulist));
    ulist *Gp = (ulist *)calloc((size_t)n, sizeof(ulist));  /* G' */
    ulist *F = (ulist *)calloc((size_t)n, sizeof(ulist));   /* final */
    ent64 *buf = (ent64 *)malloc(sizeof(ent64) * (size_t)(L + nqd + M + 2));
    uint32_t *res = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(M + 1));
    uint32_t *snap = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(M + 1));
    unsigned char *seen = (unsigned char *)calloc((size_t)n, 1);
    unsigned char *visited = (unsigned char *)malloc((size_t)n);
    unsigned char *checked = (unsigned char *)malloc((size_t)L);
    if (!B || !Gpj || !Gp || !F || !buf || !res || !snap || !seen || !visited || !checked)
        goto done;
    for (int64_t t = 0; t < nt; ++t)
        for (int32_t r = 0; r < nqd; ++r)
            if ((int64_t)knn[t * nqd + r] >= n) { rc = ORC_EINVAL; goto done; }

    /* Alg. 1, bipartite step: x = the closest base node of t gets the edge x -> t;
     * N_out(t) keeps the other nqd - 1 ids (knn row from rank 1 on). */
    for (int64_t t = 0; t < nt; ++t)
        if (ul_push(&B[knn[t * nqd]], (uint32_t)t)) goto done;

    /* Alg. 2: neighbourhood-aware projection. */
    for (int64_t xi = 0; xi < n; ++xi) {
        uint32_t x = (uint32_t)xi;
        if (B[x].n == 0) continue;
        ++pivots;
        const float *xv = X + xi * d;
        int32_t nc = 0;
        for (int32_t si = 0; si < B[x].n && nc < L; ++si) {
            const uint32_t *nout = knn + (int64_t)B[x].v[si] * nqd + 1;
            for (int32_t r = 0; r < nqd - 1 && nc < L; ++r) {
                uint32_t c = nout[r];
                if (c == x || seen[c]) continue;
                seen[c] = 1;
                buf[nc].id = c;
                buf[nc].d = cdist(prec, xv, X + (int64_t)c * d, d);
                ++nc;
            }
        }
        for (int32_t i = 0; i < nc; ++i) seen[buf[i].id] = 0;
        qsort(buf, (size_t)nc, sizeof(ent64), cmp_ent64);
        int32_t nr = acquire_neighbors(prec, X, d, x, buf, nc, M, 1, res);
        Gpj[x].n = 0;                                    /* N'(x) replaces the list */
        for (int32_t i = 0; i < nr; ++i)
            if (ul_push(&Gpj[x], res[i])) goto done;
        for (int32_t i = 0; i < nr; ++i) snap[i] = res[i];
        for (int32_t i = 0; i < nr; ++i)
            if (reverse_update(prec, X, d, Gpj, snap[i], x, M, 1, buf, res, &proj_reprunes)) goto done;
    }

    int64_t isolated = 0;
    {
        unsigned char *hasin = (unsigned char *)calloc((size_t)n, 1);
        if (!hasin) goto done;
        for (int64_t v = 0; v < n; ++v)
            for (int32_t j = 0; j < Gpj[v].n; ++j) hasin[Gpj[v].v[j]] = 1;
        for (int64_t v = 0; v < n; ++v)
            if (!hasin[v] && Gpj[v].n == 0) ++isolated;
        free(hasin);
    }

    /* Alg. 1, enhancement loop: connectivity enhancement on G' (a copy of G_pj). */
    for (int64_t v = 0; v < n; ++v)
        for (int32_t j = 0; j < Gpj[v].n; ++j)
            if (ul_push(&Gp[v], Gpj[v].v[j])) goto done;
    ent64 *pool = (ent64 *)malloc(sizeof(ent64) * (size_t)L);
    if (!pool) goto done;
    for (int64_t xi = 0; xi < n; ++xi) {
        uint32_t x = (uint32_t)xi;
        int32_t ps = beam_search_f64_lists(prec, X, n, d, Gpj, entry, X + xi * d, L, pool, checked,
                                           visited);
        int32_t nc = 0;
        for (int32_t i = 0; i < ps; ++i)
            if (pool[i].id != x) buf[nc++] = pool[i];
        int32_t nr = acquire_neighbors(prec, X, d, x, buf, nc, M, 0, res);
        Gp[x].n = 0;
        for (int32_t i = 0; i < nr; ++i)
            if (ul_push(&Gp[x], res[i])) { free(pool); goto done; }
        for (int32_t i = 0; i < nr; ++i) snap[i] = res[i];
        for (int32_t i = 0; i < nr; ++i)
            if (reverse_update(prec, X, d, Gp, snap[i], x, M, 0, buf, res, &ce_reprunes)) {
                free(pool);
                goto done;
            }
    }
    free(pool);

    /* Alg. 1, final union: N_pj(x) followed by N'(x) minus N_pj(x). */
    for (int64_t v = 0; v < n; ++v) {
        for (int32_t j = 0; j < Gpj[v].n; ++j)
            if (ul_push(&F[v], Gpj[v].v[j])) goto done;
        for (int32_t j = 0; j < Gp[v].n; ++j)
            if (!ul_has(&Gpj[v], Gp[v].v[j]))
                if (ul_push(&F[v], Gp[v].v[j])) goto done;
    }

    /* Final adjacency rows (compact, then padding), before the repair. */
    const int32_t R = 2 * M;
    int64_t pj_edges = 0;
    for (int64_t v = 0; v < n; ++v) {
        pj_edges += Gpj[v].n;
        if (pj_out)
            for (int32_t j = 0; j < M; ++j)
                pj_out[v * M + j] = j < Gpj[v].n ? Gpj[v].v[j] : ORC_NONE;
        for (int32_t j = 0; j < R; ++j)
            adj_out[v * R + j] = j < F[v].n ? F[v].v[j] : ORC_NONE;
    }
    int64_t unreachable0 = 0;
    repairs = repair_prec(prec, X, n, d, adj_out, R, entry, &unreachable0);
    if (repairs < 0) goto done;
    int64_t fin_edges = 0;
    for (int64_t v = 0; v < n * R; ++v) fin_edges += adj_out[v] != ORC_NONE;
    if (stats) {
        stats[0] = pivots;
        stats[1] = proj_reprunes;
        stats[2] = ce_reprunes;
        stats[3] = repairs;
        stats[4] = pj_edges;
        stats[5] = fin_edges;
        stats[6] = isolated;
        stats[7] = unreachable0;
    }
    rc = ORC_OK;
done:
    ul_free_all(B, n);
    ul_free_all(Gpj, n);
    ul_free_all(Gp, n);
    ul_free_all(F, n);
    free(buf);
    free(res);
    free(snap);
    free(seen);
    free(visited);
    free(checked);
    return rc;
}

int orc_build(const float *X, int64_t n, int64_t nt, int32_t d, const uint32_t *knn, int32_t nqd, int32_t M,
              int32_t L, uint32_t entry, uint32_t *pj_out, uint32_t *adj_out, int64_t *stats) {
    return orc_build_prec(X, n, nt, d, knn, nqd, M, L, entry, pj_out, adj_out, stats, 0);
}


/*
 * Insertion through the saved bipartite graph (Sec. 5.7), one new row at a
 * time in id order (rows n_old .. n_total-1 of X; their adjacency rows start
 * empty and nothing links to them, so searches cannot reach them before
 * their turn). For new row v:
 *   1. beam search (FP32, width L, visit cap max_visits) of X[v] from the
 *      entry over the current graph;
 *   2. the first pool entry b that some training query is connected to (b is
 *      in N_out(t), or b is the nearest base row (pivot) of t);
 *   3. of those queries, q = the one nearest to v (-dot_fixed, ties by id);
 *   4. projection of the sub-bipartite graph N_out(q) + q + v with v as the
 *      pivot: N(v) = Alg. 3 with fill (FP32 fixed-order distances) over
 *      N_out(q) sorted by (delta(v, c), id); when no pool entry is connected
 *      to a query, over the search pool instead;
 *   5. the edges of v merge into the graph: v's row is N(v); each p in N(v)
 *      gets p -> v, appended when its row has room, else its row and v are
 *      re-pruned to R with Alg. 3 (fill) in (delta(p, c), id) order;
 *   6. v joins N_out(q) (while N_out(q) has room) for later insertions.
 * adj [n_total][R] and nout [nt][nout_cap] / nout_cnt [nt] are updated in
 * place; chosen_q[i] is q for row n_old + i, or -1. Returns 0, 1 for bad
 * arguments, 2 when out of memory.
 */
static void sort_by_fixed_dist(const float *X, int32_t d, const float *xv, uint32_t *ids, int32_t m) {
    for (int32_t i = 1; i < m; ++i) {
        const uint32_t e = ids[i];
        const float de = -orc_dot_fixed(xv, X + (int64_t)e * d, d);
        int32_t j = i;
        while (j > 0) {
            const float dj = -orc_dot_fixed(xv, X + (int64_t)ids[j - 1] * d, d);
            if (!less_f32(de, e, dj, ids[j - 1])) break;
            ids[j] = ids[j - 1];
            --j;
        }
        ids[j] = e;
    }
}

int orc_insert(const float *X, int64_t n_total, int32_t d, uint32_t *adj, int32_t R, uint32_t entry,
               int64_t n_old, const float *T, int64_t nt, const uint32_t *pivot, uint32_t *nout,
               int32_t *nout_cnt, int32_t nout_cap, int32_t M, int32_t L, uint32_t max_visits,
               int32_t *chosen_q) {
    if (n_old < 1 || n_total < n_old || (int64_t)entry >= n_old || d < 1 || R < 1 || M < 1 || M > R ||
        L < 1 || nt < 1 || nout_cap < 1 || max_visits < 1)
        return ORC_EINVAL;
    /* queries connected to each base row: in-edges from N_out, and pivot edges */
    ulist *inc = (ulist *)calloc((size_t)n_total, sizeof(ulist));
    ent32 *pool = (ent32 *)malloc(sizeof(ent32) * (size_t)L);
    unsigned char *visited = (unsigned char *)malloc((size_t)n_total);
    float *tmp = (float *)malloc(sizeof(float) * (size_t)d);
    uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nout_cap + L + R + 1));
    uint32_t *res = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(R + 1));
    int rc = ORC_OK;
    if (!inc || !pool || !visited || !tmp || !cand || !res) { rc = ORC_ENOMEM; goto done; }
    for (int64_t t = 0; t < nt; ++t) {
        if (pivot[t] < n_total && ul_push(&inc[pivot[t]], (uint32_t)t)) { rc = ORC_ENOMEM; goto done; }
        for (int32_t j = 0; j < nout_cnt[t]; ++j) {
            const uint32_t b = nout[t * nout_cap + j];
            if (b < n_total && !ul_has(&inc[b], (uint32_t)t) && ul_push(&inc[b], (uint32_t)t)) {
                rc = ORC_ENOMEM;
                goto done;
            }
        }
    }
    for (int64_t v = n_old; v < n_total; ++v) {
        const float *xv = X + v * d;
        int32_t size = 0;
        uint32_t nv = 0, nh = 0;
        search_one(0, X, NULL, n_total, d, adj, R, entry, xv, L, max_visits, pool, &size, &nv, &nh, NULL, 0,
                   visited, tmp);
        int64_t q = -1;
        for (int32_t r = 0; r < size && q < 0; ++r) {
            const ulist *qs = &inc[pool[r].id];
            for (int32_t j = 0; j < qs->n; ++j) {
                const uint32_t t = qs->v[j];
                const float dt = -orc_dot_fixed(xv, T + (int64_t)t * d, d);
                if (q < 0 || less_f32(dt, t, -orc_dot_fixed(xv, T + q * d, d), (uint32_t)q)) q = t;
            }
        }
        int32_t nc = 0;
        if (q >= 0) {
            for (int32_t j = 0; j < nout_cnt[q]; ++j) cand[nc++] = nout[q * nout_cap + j];
            sort_by_fixed_dist(X, d, xv, cand, nc);
        } else {
            for (int32_t r = 0; r < size; ++r) cand[nc++] = pool[r].id;   /* already in (delta, id) order */
        }
        int32_t nr = orc_acquire_neighbors_f32(X, n_total, d, (uint32_t)v, cand, nc, M, 1, res);
        if (nr < 0) { rc = ORC_EINVAL; goto done; }
        uint32_t *rowv = adj + v * R;
        for (int32_t j = 0; j < R; ++j) rowv[j] = j < nr ? res[j] : ORC_NONE;
        for (int32_t j = 0; j < nr; ++j) {
            const uint32_t p = rowv[j];
            uint32_t *rp = adj + (int64_t)p * R;
            int32_t deg = 0, has = 0;
            while (deg < R && rp[deg] != ORC_NONE) { has |= rp[deg] == (uint32_t)v; ++deg; }
            if (has) continue;
            if (deg < R) { rp[deg] = (uint32_t)v; continue; }
            int32_t m = 0;
            for (int32_t t = 0; t < R; ++t) cand[m++] = rp[t];
            cand[m++] = (uint32_t)v;
            sort_by_fixed_dist(X, d, X + (int64_t)p * d, cand, m);
            const int32_t k2 = orc_acquire_neighbors_f32(X, n_total, d, p, cand, m, R, 1, res);
            for (int32_t t = 0; t < R; ++t) rp[t] = t < k2 ? res[t] : ORC_NONE;
        }
        if (q >= 0 && nout_cnt[q] < nout_cap) {
            nout[q * nout_cap + nout_cnt[q]++] = (uint32_t)v;
            if (ul_push(&inc[v], (uint32_t)q)) { rc = ORC_ENOMEM; goto done; }
        }
        chosen_q[v - n_old] = (int32_t)q;
    }
done:
    if (inc) for (int64_t i = 0; i < n_total; ++i) free(inc[i].v);
    free(inc);
    free(pool);
    free(visited);
    free(tmp);
    free(cand);
    free(res);
    return rc;
}
