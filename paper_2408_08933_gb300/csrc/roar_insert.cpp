// Insertion through the saved bipartite graph (Sec. 5.7): new base rows join
// a built RoarGraph without a rebuild. Rows n_old .. n_total-1 are inserted
// one at a time in id order; for row v:
//   1. beam search of X[v] over the current graph (GPU, roar_search, the
//      whole width-L pool, visit cap 16384);
//   2. the first pool entry b that some training query is connected to (b in
//      N_out(t), or b is t's nearest base row, its pivot);
//   3. q = the connected query nearest to v (FP32 fixed-order dot, ties by id);
//   4. N(v) = AcquireNeighbors with fill over N_out(q) (GPU, roar_acquire,
//      which sorts by (delta(v, c), id)); with no connected pool entry, over
//      the search pool;
//   5. v's row is N(v); each p in N(v) gets p -> v, appended when p's row has
//      room, else p's row and v are re-pruned to R with fill (one roar_acquire
//      launch for all such p);
//   6. v joins N_out(q) while it has room.
// Every keep / drop decision is FP32 with the search's fixed summation order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "roargraph.h"

namespace roar {
roar_status cuda_fail(cudaError_t e, const char *what);
void set_error(const char *msg);
}  // namespace roar

using namespace roar;

namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;

// <a, b> in FP32: element i accumulates (fmaf, increasing i) into lane
// (i >> 2) & 31 of 32 partial sums from +0, then s_l = s_l + s_(l xor o) for
// o = 16, 8, 4, 2, 1; lane 0 is the result (the search kernel's order).
float dot_fixed_host(const float *a, const float *b, int d) {
    float lane[32] = {0};
    for (int i = 0; i < d; ++i) lane[(i >> 2) & 31] = std::fmaf(a[i], b[i], lane[(i >> 2) & 31]);
    for (int o = 16; o >= 1; o >>= 1) {
        float next[32];
        for (int l = 0; l < 32; ++l) next[l] = lane[l] + lane[l ^ o];
        std::memcpy(lane, next, sizeof lane);
    }
    return lane[0];
}

bool less_entry(float da, uint32_t ia, float db, uint32_t ib) { return da < db || (da == db && ia < ib); }

}  // namespace

extern "C" roar_status roar_insert(const float *X_dev, int64_t n_total, int32_t d, uint32_t *adj_dev, int32_t R,
                                   uint32_t entry, int64_t n_old, const float *T_host, int64_t nt,
                                   const uint32_t *pivot_host, uint32_t *nout_host, int32_t *nout_cnt_host,
                                   int32_t nout_cap, int32_t M, int32_t L, int32_t *chosen_q_host, void *stream) {
    if (!X_dev || !adj_dev || !T_host || !pivot_host || !nout_host || !nout_cnt_host || !chosen_q_host ||
        n_old < 1 || n_total < n_old || n_total >= 0x7FFFFFFF || (int64_t)entry >= n_old || d < 4 || d % 4 ||
        d > 1024 || R < 1 || R > 64 || M < 1 || M > R || L < 1 || L > ROAR_MAX_L || nt < 1 || nout_cap < 1 ||
        nout_cap > 1024) {
        set_error("roar_insert: bad arguments (need n_old >= 1, entry < n_old, d % 4 == 0, 1 <= M <= R <= 64, "
                  "L <= ROAR_MAX_L, nout_cap <= 1024)");
        return ROAR_EINVAL;
    }
    if (n_total == n_old) return ROAR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_new = n_total - n_old;
    std::vector<uint32_t> adj((size_t)n_total * R);
    std::vector<float> Xnew((size_t)n_new * d);
    cudaError_t e = cudaMemcpyAsync(adj.data(), adj_dev, adj.size() * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(Xnew.data(), X_dev + (size_t)n_old * d, Xnew.size() * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "roar_insert: copy graph");
    // queries connected to each base row
    std::vector<std::vector<uint32_t>> inc((size_t)n_total);
    for (int64_t t = 0; t < nt; ++t) {
        if (pivot_host[t] < n_total) inc[pivot_host[t]].push_back((uint32_t)t);
        for (int j = 0; j < nout_cnt_host[t]; ++j) {
            const uint32_t b = nout_host[t * nout_cap + j];
            if (b < n_total && std::find(inc[b].begin(), inc[b].end(), (uint32_t)t) == inc[b].end())
                inc[b].push_back((uint32_t)t);
        }
    }
    const int CS = std::max(std::max(nout_cap, L), R + 1);   // candidate row width
    uint32_t *ids = nullptr, *cand = nullptr, *xs = nullptr, *out = nullptr;
    float *dist = nullptr;
    int32_t *nc = nullptr, *cnt = nullptr;
    e = cudaMalloc(&ids, (size_t)L * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dist, (size_t)L * 4);
    if (e == cudaSuccess) e = cudaMalloc(&cand, (size_t)(M + 1) * CS * 4);
    if (e == cudaSuccess) e = cudaMalloc(&xs, (size_t)(M + 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&nc, (size_t)(M + 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)(M + 1) * R * 4);
    if (e == cudaSuccess) e = cudaMalloc(&cnt, (size_t)(M + 1) * 4);
    roar_status rc = ROAR_OK;
    roar_index *gi = nullptr;
    if (e == cudaSuccess) rc = roar_index_create(n_total, d, X_dev, ROAR_F32, nullptr, nullptr, adj_dev, R, entry,
                                                 16384u, &gi);
    // One query at a time: its latency is the cost, so search with a team of
    // 8 warps per query (same results as one warp, shorter hops).
    if (e == cudaSuccess && rc == ROAR_OK) rc = roar_index_set_tuning(gi, L, 8, 0, 0);
    std::vector<uint32_t> hid((size_t)L), hc((size_t)(M + 1) * CS), hout((size_t)(M + 1) * R), hx((size_t)M + 1);
    std::vector<int32_t> hnc((size_t)M + 1), hcnt((size_t)M + 1);
    for (int64_t v = n_old; e == cudaSuccess && rc == ROAR_OK && v < n_total; ++v) {
        const float *xv = Xnew.data() + (size_t)(v - n_old) * d;
        // 1. search
        rc = roar_search(gi, X_dev + (size_t)v * d, 1, L, L, ids, dist, nullptr, nullptr, nullptr, stream);
        if (rc != ROAR_OK) break;
        e = cudaMemcpyAsync(hid.data(), ids, (size_t)L * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        // 2-3. the nearest query connected to the first connected pool entry
        int64_t q = -1;
        float qd = 0.0f;
        for (int r = 0; r < L && q < 0 && hid[r] != kNone; ++r) {
            for (uint32_t t : inc[hid[r]]) {
                const float dt = -dot_fixed_host(xv, T_host + (size_t)t * d, d);
                if (q < 0 || less_entry(dt, t, qd, (uint32_t)q)) {
                    q = t;
                    qd = dt;
                }
            }
        }
        // 4. N(v) by Alg. 3 with fill
        int m = 0;
        if (q >= 0)
            for (int j = 0; j < nout_cnt_host[q]; ++j) hc[m++] = nout_host[q * nout_cap + j];
        else
            for (int r = 0; r < L && hid[r] != kNone; ++r) hc[m++] = hid[r];
        std::fill(hc.begin() + m, hc.begin() + CS, kNone);
        hx[0] = (uint32_t)v;
        hnc[0] = m;
        e = cudaMemcpyAsync(cand, hc.data(), (size_t)CS * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(xs, hx.data(), 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(nc, hnc.data(), 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        rc = roar_acquire(X_dev, n_total, d, xs, 1, cand, CS, nc, M, 1, out, cnt, nullptr, stream);
        if (rc != ROAR_OK) break;
        e = cudaMemcpyAsync(hout.data(), out, (size_t)M * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hcnt.data(), cnt, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        if (hcnt[0] < 0) {
            set_error("roar_insert: an id outside the base set");
            rc = ROAR_EINVAL;
            break;
        }
        const int nr = hcnt[0];
        uint32_t *rowv = adj.data() + (size_t)v * R;
        for (int j = 0; j < R; ++j) rowv[j] = j < nr ? hout[j] : kNone;
        // 5. reverse edges: append where there is room, re-prune full rows
        std::vector<int64_t> changed{v}, full;
        for (int j = 0; j < nr; ++j) {
            const uint32_t p = rowv[j];
            uint32_t *rp = adj.data() + (size_t)p * R;
            int deg = 0;
            bool has = false;
            while (deg < R && rp[deg] != kNone) has |= rp[deg++] == (uint32_t)v;
            if (has) continue;
            changed.push_back(p);
            if (deg < R) rp[deg] = (uint32_t)v;
            else full.push_back(p);
        }
        if (!full.empty()) {
            const int nf = (int)full.size();
            for (int i = 0; i < nf; ++i) {
                uint32_t *r = hc.data() + (size_t)i * CS;
                std::copy(adj.data() + (size_t)full[i] * R, adj.data() + (size_t)full[i] * R + R, r);
                r[R] = (uint32_t)v;
                std::fill(r + R + 1, r + CS, kNone);
                hx[i] = (uint32_t)full[i];
                hnc[i] = R + 1;
            }
            e = cudaMemcpyAsync(cand, hc.data(), (size_t)nf * CS * 4, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(xs, hx.data(), (size_t)nf * 4, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(nc, hnc.data(), (size_t)nf * 4, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) break;
            rc = roar_acquire(X_dev, n_total, d, xs, nf, cand, CS, nc, R, 1, out, cnt, nullptr, stream);
            if (rc != ROAR_OK) break;
            e = cudaMemcpyAsync(hout.data(), out, (size_t)nf * R * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hcnt.data(), cnt, (size_t)nf * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) break;
            for (int i = 0; i < nf; ++i) {
                uint32_t *rp = adj.data() + (size_t)full[i] * R;
                for (int t = 0; t < R; ++t) rp[t] = t < hcnt[i] ? hout[(size_t)i * R + t] : kNone;
            }
        }
        for (int64_t p : changed) {
            e = cudaMemcpyAsync(adj_dev + (size_t)p * R, adj.data() + (size_t)p * R, (size_t)R * 4,
                                cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) break;
        }
        if (e != cudaSuccess) break;
        // 6. the bipartite graph learns v
        if (q >= 0 && nout_cnt_host[q] < nout_cap) {
            nout_host[q * nout_cap + nout_cnt_host[q]++] = (uint32_t)v;
            inc[v].push_back((uint32_t)q);
        }
        chosen_q_host[v - n_old] = (int32_t)q;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    roar_index_destroy(gi);
    cudaFree(ids);
    cudaFree(dist);
    cudaFree(cand);
    cudaFree(xs);
    cudaFree(nc);
    cudaFree(out);
    cudaFree(cnt);
    if (e != cudaSuccess) return cuda_fail(e, "roar_insert");
    return rc;
}
