// C ABI entry points of libroargraph: handle management and search launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "roar_internal.cuh"

namespace roar {

static thread_local char g_last_error[256] = "";

roar_status cuda_fail(cudaError_t e, const char *what) {
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s", what, cudaGetErrorString(e));
    return ROAR_ECUDA;
}

void set_error(const char *msg) { std::snprintf(g_last_error, sizeof g_last_error, "%s", msg); }

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

int next_pow2_log2(uint64_t x) {
    int lg = 0;
    while ((1ull << lg) < x) ++lg;
    return lg;
}

}  // namespace roar

using namespace roar;

struct roar_index {
    int64_t n;
    int32_t d;
    roar_dtype dtype;
    const float *base32;
    const void *trav;
    const float *scales;
    const uint32_t *adj;
    const uint32_t *tomb = nullptr;  // caller-owned deletion bitmap or null
    // Bipartite graph G_bi (null for a plain graph): `adj` holds N_out rows of
    // bi_nt query nodes, B(x) = bi_q[bi_off[x] .. bi_off[x + 1]).
    const int64_t *bi_off = nullptr;
    const uint32_t *bi_q = nullptr;
    int64_t bi_nt = 0;
    int32_t rmax;
    uint32_t entry;
    uint32_t max_visits;
    int device;
    int num_sms;
    // Launch tuning per beam-width bucket (L <= 32, 64, ..., 1024):
    // warps per query team, visited-table mode (0 auto, -1 bitmap only,
    // 5..15 shared slots log2), resident-CTA cap per SM (0 = occupancy limit).
    struct Tune {
        int tw = 1;
        int hash = 0;
        int bps_cap = 0;
    } tune[6];
    // scratch: one visited bitmap + log per resident warp, grown on demand
    uint32_t *vbits = nullptr;
    uint32_t *vlog = nullptr;
    int64_t vslots = 0;
    int64_t vbits_words = 0;
    int32_t vlog_cap = 0;
    unsigned int *work = nullptr;
    // device staging for roar_search_host, grown on demand
    unsigned char *stage = nullptr;
    size_t stage_bytes = 0;
    std::mutex mu;
};

extern "C" const char *roar_status_string(roar_status s) {
    switch (s) {
        case ROAR_OK: return "ok";
        case ROAR_EINVAL: return "invalid argument";
        case ROAR_ENOMEM: return "out of memory";
        case ROAR_ECUDA: return "CUDA error";
        case ROAR_EOVERFLOW: return "visit cap reached";
        case ROAR_ETIMEOUT: return "timed out";
        case ROAR_EBUSY: return "busy";
    }
    return "unknown status";
}

extern "C" const char *roar_last_error(void) { return g_last_error; }

extern "C" roar_status roar_index_create(int64_t n, int32_t d, const float *base_f32,
                                         roar_dtype trav_dtype, const void *base_trav,
                                         const float *scales, const uint32_t *adj, int32_t rmax,
                                         uint32_t entry, uint32_t max_visits, roar_index **out) {
    if (!out) return ROAR_EINVAL;
    *out = nullptr;
    if (n < 1 || n >= (int64_t)kIdMask || d < 4 || d > 1024 || d % 4 != 0 || !base_f32 || !adj ||
        rmax < 1 || rmax > ROAR_MAX_RMAX || (int64_t)entry >= n) {
        set_error("roar_index_create: bad size, pointer or entry");
        return ROAR_EINVAL;
    }
    if (!aligned(base_f32, 16) || !aligned(adj, 4)) {
        set_error("roar_index_create: base_f32 must be 16-byte and adj 4-byte aligned");
        return ROAR_EINVAL;
    }
    switch (trav_dtype) {
        case ROAR_F32:
            if (base_trav || scales) {
                set_error("roar_index_create: ROAR_F32 takes no copy and no scales");
                return ROAR_EINVAL;
            }
            break;
        case ROAR_BF16:
            if (!base_trav || !aligned(base_trav, 8) || scales) {
                set_error("roar_index_create: ROAR_BF16 needs an 8-byte aligned copy, no scales");
                return ROAR_EINVAL;
            }
            break;
        case ROAR_FP8_E4M3:
            if (!base_trav || !aligned(base_trav, 4) || !scales || !aligned(scales, 4)) {
                set_error("roar_index_create: ROAR_FP8_E4M3 needs a 4-byte aligned copy and scales");
                return ROAR_EINVAL;
            }
            break;
        default:
            set_error("roar_index_create: unknown dtype");
            return ROAR_EINVAL;
    }
    if (max_visits == 0) max_visits = 16384u;
    if (max_visits > (1u << 24)) {
        set_error("roar_index_create: max_visits above 2^24");
        return ROAR_EINVAL;
    }
    roar_index *idx = new (std::nothrow) roar_index();
    if (!idx) return ROAR_ENOMEM;
    idx->n = n;
    idx->d = d;
    idx->dtype = trav_dtype;
    idx->base32 = base_f32;
    idx->trav = trav_dtype == ROAR_F32 ? (const void *)base_f32 : base_trav;
    idx->scales = scales;
    idx->adj = adj;
    idx->rmax = rmax;
    idx->entry = entry;
    idx->max_visits = max_visits;
    idx->vbits_words = (n + 31) / 32;
    idx->vlog_cap = (int32_t)max_visits + ROAR_MAX_RMAX;
    cudaError_t e = cudaGetDevice(&idx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&idx->num_sms, cudaDevAttrMultiProcessorCount, idx->device);
    if (e == cudaSuccess) e = cudaMalloc(&idx->work, sizeof(unsigned int));
    if (e != cudaSuccess) {
        roar_status st = cuda_fail(e, "roar_index_create");
        delete idx;
        return st;
    }
    *out = idx;
    return ROAR_OK;
}

extern "C" roar_status roar_index_create_bipartite(int64_t n, int32_t d, const float *base_f32,
                                                   const uint32_t *nout, int32_t rn, int64_t nt,
                                                   const int64_t *bi_off, const uint32_t *bi_q, uint32_t entry,
                                                   uint32_t max_visits, roar_index **out) {
    if (!out) return ROAR_EINVAL;
    *out = nullptr;
    if (nt < 1 || nt >= (int64_t)kIdMask || !bi_off || !bi_q || !aligned(bi_off, 8) || !aligned(bi_q, 4)) {
        set_error("roar_index_create_bipartite: bad query-node count or CSR arrays");
        return ROAR_EINVAL;
    }
    roar_index *idx = nullptr;
    roar_status st = roar_index_create(n, d, base_f32, ROAR_F32, nullptr, nullptr, nout, rn, entry, max_visits, &idx);
    if (st != ROAR_OK) return st;
    idx->bi_off = bi_off;
    idx->bi_q = bi_q;
    idx->bi_nt = nt;
    *out = idx;
    return ROAR_OK;
}

extern "C" roar_status roar_index_set_hash_log2(roar_index *idx, int32_t log2) {
    if (!idx || (log2 != 0 && log2 != -1 && (log2 < 5 || log2 > 15))) {
        set_error("roar_index_set_hash_log2: log2 must be 0, -1 or in [5, 15]");
        return ROAR_EINVAL;
    }
    std::lock_guard<std::mutex> lock(idx->mu);
    for (auto &t : idx->tune) t.hash = log2;
    return ROAR_OK;
}

extern "C" roar_status roar_index_set_tombstones(roar_index *idx, const uint32_t *bits) {
    if (!idx || (bits && !aligned(bits, 4))) {
        set_error("roar_index_set_tombstones: bad handle or bitmap pointer");
        return ROAR_EINVAL;
    }
    std::lock_guard<std::mutex> lock(idx->mu);
    idx->tomb = bits;
    return ROAR_OK;
}

extern "C" void roar_index_destroy(roar_index *idx) {
    if (!idx) return;
    cudaDeviceSynchronize();
    cudaFree(idx->vbits);
    cudaFree(idx->vlog);
    cudaFree(idx->work);
    cudaFree(idx->stage);
    delete idx;
}

namespace roar {

// Make room for `slots` visited bitmaps and logs (synchronises the device when it grows).
static roar_status ensure_scratch(roar_index *idx, int64_t slots) {
    if (slots <= idx->vslots) return ROAR_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "ensure_scratch");
    cudaFree(idx->vbits);
    cudaFree(idx->vlog);
    idx->vbits = nullptr;
    idx->vlog = nullptr;
    idx->vslots = 0;
    const size_t bb = (size_t)slots * idx->vbits_words * sizeof(uint32_t);
    e = cudaMalloc(&idx->vbits, bb);
    if (e == cudaSuccess) e = cudaMalloc(&idx->vlog, (size_t)slots * idx->vlog_cap * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(idx->vbits, 0, bb);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(idx->vbits);
        cudaFree(idx->vlog);
        idx->vbits = nullptr;
        idx->vlog = nullptr;
        cudaGetLastError();
        set_error("roar_search: cannot allocate the visited bitmaps");
        return ROAR_ENOMEM;
    }
    idx->vslots = slots;
    return ROAR_OK;
}

int tune_bucket(int L) {
    int b = 0;
    while (b < 5 && (32 << b) < L) ++b;
    return b;
}

// Fill a SearchArgs for the handle and pick the launch shape.
roar_status plan_search(roar_index *idx, int32_t lmax, SearchArgs &a, int &blocks, int &tw, int64_t nq) {
    std::memset(&a, 0, sizeof a);
    const roar_index::Tune &t = idx->tune[tune_bucket(lmax)];
    a.trav = idx->trav;
    a.scales = idx->scales;
    a.base32 = idx->base32;
    a.adj = idx->adj;
    a.tomb = idx->tomb;
    a.n = idx->n;
    a.d = idx->d;
    a.rmax = idx->rmax;
    a.entry = idx->entry;
    a.dtype = (int32_t)idx->dtype;
    a.lcap = (lmax + 31) / 32 * 32;
    a.max_visits = idx->max_visits;
    a.hash_log2 = t.hash == 0 ? hash_log2_for(lmax) : (t.hash < 0 ? 0 : t.hash);
    a.bi_off = idx->bi_off;
    a.bi_q = idx->bi_q;
    a.bi_nt = idx->bi_nt;
    const bool bi = idx->bi_off != nullptr;
    tw = t.tw;
    if (bi && tw != 1) {
        set_error("roar_search: the bipartite-graph search runs one warp per query");
        return ROAR_EINVAL;
    }
    int bps = search_blocks_per_sm((int)idx->dtype, idx->d, idx->rmax, a.lcap, a.hash_log2, tw, bi);
    if (bps <= 0) {
        set_error("roar_search: this L does not fit in shared memory");
        return ROAR_EINVAL;
    }
    if (t.bps_cap > 0 && bps > t.bps_cap) bps = t.bps_cap;
    const int tpb = teams_per_block(tw);
    int64_t want = (nq + tpb - 1) / tpb;
    int64_t full = (int64_t)bps * idx->num_sms;
    blocks = (int)std::max<int64_t>(1, std::min(want, full));
    roar_status st = ensure_scratch(idx, full * tpb);
    if (st != ROAR_OK) return st;
    a.vbits = idx->vbits;
    a.vbits_words = idx->vbits_words;
    a.vlog = idx->vlog;
    a.vlog_cap = idx->vlog_cap;
    a.work = idx->work;
    return ROAR_OK;
}

}  // namespace roar

extern "C" roar_status roar_search(roar_index *idx, const float *queries, int64_t nq, int32_t k,
                                   int32_t L, uint32_t *ids, float *dist, uint32_t *visits,
                                   uint32_t *hops, int32_t *qstatus, void *stream) {
    if (!idx || nq < 0 || k < 1 || L < k || L > ROAR_MAX_L) {
        set_error("roar_search: need 1 <= k <= L <= ROAR_MAX_L and nq >= 0");
        return ROAR_EINVAL;
    }
    if (nq == 0) return ROAR_OK;
    if (nq >= (int64_t)1 << 31 || !queries || !ids || !dist || !aligned(queries, 16)) {
        set_error("roar_search: bad query or output pointer");
        return ROAR_EINVAL;
    }
    std::lock_guard<std::mutex> lock(idx->mu);
    SearchArgs a;
    int blocks = 0, tw = 1;
    roar_status st = plan_search(idx, L, a, blocks, tw, nq);
    if (st != ROAR_OK) return st;
    a.q = queries;
    a.nq = nq;
    a.k = k;
    a.L = L;
    a.ids = ids;
    a.dist = dist;
    a.visits = visits;
    a.hops = hops;
    a.qstatus = qstatus;
    cudaError_t e = launch_search(a, blocks, tw, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "roar_search launch");
    return ROAR_OK;
}

extern "C" roar_status roar_search_host(roar_index *idx, const float *queries_host, int64_t nq,
                                        int32_t k, int32_t L, uint32_t *ids_host, float *dist_host,
                                        uint32_t *visits_host, uint32_t *hops_host,
                                        int32_t *qstatus_host, void *stream) {
    if (!idx || nq < 0 || k < 1 || L < k || L > ROAR_MAX_L) {
        set_error("roar_search_host: need 1 <= k <= L <= ROAR_MAX_L and nq >= 0");
        return ROAR_EINVAL;
    }
    if (nq == 0) return ROAR_OK;
    if (!queries_host || !ids_host || !dist_host) return ROAR_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t qb = (size_t)nq * idx->d * sizeof(float);
    const size_t rb = (size_t)nq * k * sizeof(uint32_t);
    const size_t sb = (size_t)nq * sizeof(uint32_t);
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t need = up(qb) + 2 * up(rb) + 3 * up(sb);
    {
        std::lock_guard<std::mutex> lock(idx->mu);
        if (need > idx->stage_bytes) {
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(e, "roar_search_host");
            cudaFree(idx->stage);
            idx->stage = nullptr;
            idx->stage_bytes = 0;
            e = cudaMalloc(&idx->stage, need);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return ROAR_ENOMEM;
            }
            idx->stage_bytes = need;
        }
    }
    unsigned char *p = idx->stage;
    float *dq = (float *)p;
    p += up(qb);
    uint32_t *di = (uint32_t *)p;
    p += up(rb);
    float *dd = (float *)p;
    p += up(rb);
    uint32_t *dv = (uint32_t *)p;
    p += up(sb);
    uint32_t *dh = (uint32_t *)p;
    p += up(sb);
    int32_t *ds = (int32_t *)p;
    cudaError_t e = cudaMemcpyAsync(dq, queries_host, qb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "roar_search_host H2D");
    roar_status st = roar_search(idx, dq, nq, k, L, di, dd, dv, dh, ds, stream);
    if (st != ROAR_OK) return st;
    e = cudaMemcpyAsync(ids_host, di, rb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dist_host, dd, rb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && visits_host) e = cudaMemcpyAsync(visits_host, dv, sb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && hops_host) e = cudaMemcpyAsync(hops_host, dh, sb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && qstatus_host) e = cudaMemcpyAsync(qstatus_host, ds, sb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "roar_search_host D2H");
    return ROAR_OK;
}

// ---------------------------------------------------------------------------
// Uneven batches, CUDA-graph plans and the launch autotuner.
// ---------------------------------------------------------------------------

namespace roar {

static roar_status fill_uneven(roar_index *idx, const float *queries, int64_t nq, const int32_t *k_dev,
                               const int32_t *L_dev, const int64_t *out_off, int32_t L_max,
                               const int32_t *order, uint32_t *ids, float *dist, uint32_t *visits,
                               uint32_t *hops, int32_t *qstatus, SearchArgs &a, int &blocks, int &tw) {
    if (!idx || nq < 0 || L_max < 1 || L_max > ROAR_MAX_L) {
        set_error("roar_search_uneven: need 1 <= L_max <= ROAR_MAX_L and nq >= 0");
        return ROAR_EINVAL;
    }
    if (nq == 0) return ROAR_OK;
    if (nq >= (int64_t)1 << 31 || !queries || !k_dev || !L_dev || !out_off || !ids || !dist ||
        !aligned(queries, 16)) {
        set_error("roar_search_uneven: bad pointer");
        return ROAR_EINVAL;
    }
    roar_status st = plan_search(idx, L_max, a, blocks, tw, nq);
    if (st != ROAR_OK) return st;
    a.q = queries;
    a.nq = nq;
    a.k_arr = k_dev;
    a.L_arr = L_dev;
    a.out_off = out_off;
    a.order = order;
    a.ids = ids;
    a.dist = dist;
    a.visits = visits;
    a.hops = hops;
    a.qstatus = qstatus;
    return ROAR_OK;
}

}  // namespace roar

extern "C" roar_status roar_search_uneven(roar_index *idx, const float *queries, int64_t nq,
                                          const int32_t *k_dev, const int32_t *L_dev,
                                          const int64_t *out_off, int32_t L_max, const int32_t *order,
                                          uint32_t *ids, float *dist, uint32_t *visits, uint32_t *hops,
                                          int32_t *qstatus, void *stream) {
    if (!idx) return ROAR_EINVAL;
    if (nq == 0) return ROAR_OK;
    std::lock_guard<std::mutex> lock(idx->mu);
    SearchArgs a;
    int blocks = 0, tw = 1;
    roar_status st = fill_uneven(idx, queries, nq, k_dev, L_dev, out_off, L_max, order, ids, dist,
                                 visits, hops, qstatus, a, blocks, tw);
    if (st != ROAR_OK || nq == 0) return st;
    cudaError_t e = launch_search(a, blocks, tw, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "roar_search_uneven launch");
    return ROAR_OK;
}

struct roar_plan {
    roar_index *idx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t *order = nullptr;  // owned processing order (longest beam first), or null
};

extern "C" roar_status roar_plan_create(roar_index *idx, const float *queries, int64_t nq,
                                        const int32_t *k_dev, const int32_t *L_dev,
                                        const int64_t *out_off, int32_t L_max, int32_t longest_first,
                                        uint32_t *ids, float *dist, uint32_t *visits, uint32_t *hops,
                                        int32_t *qstatus, void *stream, roar_plan **out) {
    if (!out || !idx || nq < 1) return ROAR_EINVAL;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    roar_plan *p = new (std::nothrow) roar_plan();
    if (!p) return ROAR_ENOMEM;
    p->idx = idx;
    cudaError_t e = cudaSuccess;
    if (longest_first) {
        // Longest beams first (LPT order) keeps the persistent launch's tail short.
        std::vector<int32_t> Lh((size_t)nq), ord((size_t)nq);
        e = cudaMemcpyAsync(Lh.data(), L_dev, (size_t)nq * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) {
            std::iota(ord.begin(), ord.end(), 0);
            std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return Lh[x] > Lh[y]; });
            e = cudaMalloc(&p->order, (size_t)nq * 4);
        }
        if (e == cudaSuccess) e = cudaMemcpy(p->order, ord.data(), (size_t)nq * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(p->order);
            delete p;
            return cuda_fail(e, "roar_plan_create: order");
        }
    }
    std::lock_guard<std::mutex> lock(idx->mu);
    SearchArgs a;
    int blocks = 0, tw = 1;
    roar_status st = fill_uneven(idx, queries, nq, k_dev, L_dev, out_off, L_max, p->order, ids, dist,
                                 visits, hops, qstatus, a, blocks, tw);
    if (st == ROAR_OK) {
        // Capture on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); replays go to the caller's stream.
        cudaStream_t cs = nullptr;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = launch_search(a, blocks, tw, cs, false);
            e = cudaStreamEndCapture(cs, &p->graph);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
        if (cs) cudaStreamDestroy(cs);
        if (e != cudaSuccess) st = cuda_fail(e, "roar_plan_create: capture");
    }
    if (st != ROAR_OK) {
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        cudaFree(p->order);
        delete p;
        return st;
    }
    *out = p;
    return ROAR_OK;
}

extern "C" roar_status roar_plan_launch(roar_plan *p, void *stream) {
    if (!p || !p->exec) return ROAR_EINVAL;
    cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? ROAR_OK : cuda_fail(e, "roar_plan_launch");
}

extern "C" void roar_plan_destroy(roar_plan *p) {
    if (!p) return;
    cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    cudaFree(p->order);
    delete p;
}

extern "C" roar_status roar_index_set_tuning(roar_index *idx, int32_t L, int32_t team_warps,
                                             int32_t hash_log2, int32_t blocks_per_sm_cap) {
    if (!idx || L < 1 || L > ROAR_MAX_L ||
        !(team_warps == 1 || team_warps == 2 || team_warps == 4 || team_warps == 8) ||
        (hash_log2 != 0 && hash_log2 != -1 && (hash_log2 < 5 || hash_log2 > 15)) || blocks_per_sm_cap < 0) {
        set_error("roar_index_set_tuning: bad arguments");
        return ROAR_EINVAL;
    }
    std::lock_guard<std::mutex> lock(idx->mu);
    auto &t = idx->tune[tune_bucket(L)];
    t.tw = team_warps;
    t.hash = hash_log2;
    t.bps_cap = blocks_per_sm_cap;
    return ROAR_OK;
}

extern "C" roar_status roar_autotune(roar_index *idx, const float *queries, int64_t nq, int32_t k,
                                     int32_t L, int32_t repeats, float *results, int32_t *best,
                                     void *stream) {
    // Candidate grid: team warps x visited-table mode; results gets
    // [4 x 4] milliseconds per search (inf where a variant cannot launch).
    static const int tws[4] = {1, 2, 4, 8};
    static const int hashes[4] = {0, -1, 10, 12};
    if (!idx || !queries || nq < 1 || k < 1 || L < k || L > ROAR_MAX_L || repeats < 1) return ROAR_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *ids = nullptr;
    float *dist = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&ids, (size_t)nq * k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dist, (size_t)nq * k * 4);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaFree(ids);
        cudaFree(dist);
        return cuda_fail(e, "roar_autotune");
    }
    const int b = tune_bucket(L);
    const roar_index::Tune saved = idx->tune[b];
    float best_ms = 1e30f;
    int best_i = -1;
    roar_status rc = ROAR_OK;
    for (int i = 0; i < 16 && rc == ROAR_OK; ++i) {
        idx->tune[b].tw = tws[i / 4];
        idx->tune[b].hash = hashes[i % 4];
        idx->tune[b].bps_cap = 0;
        float ms = 1e30f;
        roar_status st = roar_search(idx, queries, nq, k, L, ids, dist, nullptr, nullptr, nullptr, stream);
        if (st == ROAR_OK) {
            cudaEventRecord(e0, s);
            for (int r = 0; r < repeats && st == ROAR_OK; ++r)
                st = roar_search(idx, queries, nq, k, L, ids, dist, nullptr, nullptr, nullptr, stream);
            cudaEventRecord(e1, s);
            e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) rc = cuda_fail(e, "roar_autotune");
            else if (st == ROAR_OK) {
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= repeats;
            }
        } else if (st != ROAR_EINVAL) {
            rc = st;
        }
        if (results) results[i] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best_i = i;
        }
    }
    if (best_i >= 0) {
        idx->tune[b].tw = tws[best_i / 4];
        idx->tune[b].hash = hashes[best_i % 4];
        idx->tune[b].bps_cap = 0;
    } else {
        idx->tune[b] = saved;
    }
    if (best) *best = best_i;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(ids);
    cudaFree(dist);
    return rc;
}
