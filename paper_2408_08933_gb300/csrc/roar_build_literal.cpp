// RoarGraph construction in the literal order of Alg. 1 (Sec. 4.2), built from
// the library's GPU parts. It exists to check those parts against the steps
// the paper prints; roar_build_index is the fast, batched form.
//   bipartite step: B(x) = every training query whose nearest base row is x;
//   projection (Alg. 2): pivots in ascending id, each N'(x) = Alg. 3 with fill
//      over the per-element candidate list, replacing x's list, then each
//      reverse edge appended when there is room, else the target's list and
//      the new edge re-pruned with Alg. 3 with fill, one pivot after another;
//   enhancement: every base row searched over the fixed G_pj (GPU, roar_search,
//      width L_build) and N'(x) = Alg. 3 without fill over the result (GPU,
//      roar_acquire), then, in ascending x, x's list in G' replaced by N'(x) and
//      the reverse edges added as in projection but without fill;
//   final union: N_pj(x) followed by G'(x) minus N_pj(x);
//   repair: while a node is unreachable from the entry, the smallest such u
//      gets an edge from the nearest reachable node with a free slot, or when
//      all are full the nearest gives up its last edge.
// Every decision takes the search's fixed-order FP32 distance (element i in
// lane (i >> 2) & 31, fmaf in increasing i, butterfly o = 16 .. 1), ties by
// id. The sequential steps run on one host thread: meant for checking on
// small inputs, not for large builds.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "roargraph.h"

namespace roar {
roar_status cuda_fail(cudaError_t e, const char *what);
void set_error(const char *msg);
}  // namespace roar

using namespace roar;

namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;
using Cand = std::pair<float, uint32_t>;  // (distance, id)

float dot_fixed(const float *a, const float *b, int d) {
    float lane[32] = {0};
    for (int i = 0; i < d; ++i) lane[(i >> 2) & 31] = std::fmaf(a[i], b[i], lane[(i >> 2) & 31]);
    for (int o = 16; o >= 1; o >>= 1) {
        float next[32];
        for (int l = 0; l < 32; ++l) next[l] = lane[l] + lane[l ^ o];
        std::memcpy(lane, next, sizeof lane);
    }
    return lane[0];
}

inline float dist(const std::vector<float> &X, int d, uint32_t a, uint32_t b) {
    return -dot_fixed(X.data() + (size_t)a * d, X.data() + (size_t)b * d, d);
}

inline bool cand_less(const Cand &a, const Cand &b) {
    return a.first < b.first || (a.first == b.first && a.second < b.second);
}

// Alg. 3 over C sorted by (distance to x, id): the first candidate, then each
// candidate closer to x than to every kept one (strict), up to M; with fill,
// the remaining candidates in order up to M. x itself and repeats are skipped.
int acquire(const std::vector<float> &X, int d, uint32_t x, const std::vector<Cand> &C, int M, bool fill,
            std::vector<uint32_t> &res) {
    res.clear();
    for (size_t i = 0; i < C.size() && (int)res.size() < M; ++i) {
        const uint32_t c = C[i].second;
        if (c == x || std::find(res.begin(), res.end(), c) != res.end()) continue;
        if (res.empty()) {
            res.push_back(c);
            continue;
        }
        bool keep = true;
        for (size_t j = 0; j < res.size() && keep; ++j)
            if (!(C[i].first < dist(X, d, c, res[j]))) keep = false;
        if (keep) res.push_back(c);
    }
    if (fill)
        for (size_t i = 0; i < C.size() && (int)res.size() < M; ++i) {
            const uint32_t c = C[i].second;
            if (c != x && std::find(res.begin(), res.end(), c) == res.end()) res.push_back(c);
        }
    return (int)res.size();
}

// p gets the edge p -> x: skipped when present, appended when p's list has
// room, else p's list and x re-pruned with Alg. 3.
void reverse_update(const std::vector<float> &X, int d, std::vector<std::vector<uint32_t>> &G, uint32_t p,
                    uint32_t x, int M, bool fill, std::vector<uint32_t> &tmp) {
    auto &lp = G[p];
    if (std::find(lp.begin(), lp.end(), x) != lp.end()) return;
    if ((int)lp.size() < M) {
        lp.push_back(x);
        return;
    }
    std::vector<Cand> C;
    C.reserve(lp.size() + 1);
    for (uint32_t u : lp) C.emplace_back(dist(X, d, p, u), u);
    C.emplace_back(dist(X, d, p, x), x);
    std::sort(C.begin(), C.end(), cand_less);
    acquire(X, d, p, C, M, fill, tmp);
    lp = tmp;
}

}  // namespace

extern "C" roar_status roar_build_index_literal(const float *X_dev, int64_t n, int32_t d, const float *T_dev,
                                                int64_t nt, int32_t nq_depth, int32_t M, int32_t L_build,
                                                uint32_t *adj_dev, uint32_t *pj_dev, uint32_t *entry_out,
                                                double *stats, void *stream) {
    if (!X_dev || !T_dev || !adj_dev || !entry_out || n < 2 || n > (1 << 24) || nt < 1 || d < 8 || d % 8 ||
        d > 512 || nq_depth < 2 || nq_depth > 128 || nq_depth > n || M < 1 || 2 * M > ROAR_MAX_RMAX ||
        L_build < M || L_build > ROAR_MAX_L) {
        set_error("roar_build_index_literal: bad arguments");
        return ROAR_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const auto t_all = std::chrono::steady_clock::now();
    const int R = 2 * M;
    std::vector<float> X((size_t)n * d);
    cudaError_t e = cudaMemcpyAsync(X.data(), X_dev, X.size() * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "roar_build_index_literal: copy X");
    uint32_t entry = 0;
    roar_status rc = roar_medoid(X.data(), n, d, 0, &entry);
    if (rc != ROAR_OK) return rc;

    // Training queries' N_q nearest base rows (GPU).
    std::vector<uint32_t> knn((size_t)nt * nq_depth);
    {
        uint32_t *ki = nullptr;
        float *kd = nullptr;
        e = cudaMalloc(&ki, knn.size() * 4);
        if (e == cudaSuccess) e = cudaMalloc(&kd, knn.size() * 4);
        if (e == cudaSuccess) rc = roar_knn(T_dev, nt, X_dev, n, d, nq_depth, ki, kd, stream);
        if (e == cudaSuccess && rc == ROAR_OK) {
            e = cudaMemcpyAsync(knn.data(), ki, knn.size() * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        cudaFree(ki);
        cudaFree(kd);
        if (e != cudaSuccess) return cuda_fail(e, "roar_build_index_literal: kNN");
        if (rc != ROAR_OK) return rc;
    }
    // Bipartite step: B(x), queries in ascending id.
    std::vector<std::vector<uint32_t>> B((size_t)n);
    for (int64_t t = 0; t < nt; ++t) B[knn[(size_t)t * nq_depth]].push_back((uint32_t)t);

    // Projection (Alg. 2), pivots in ascending id.
    std::vector<std::vector<uint32_t>> pj((size_t)n);
    std::vector<unsigned char> seen((size_t)n, 0);
    std::vector<uint32_t> res, tmp, snap;
    int64_t pivots = 0;
    for (int64_t xi = 0; xi < n; ++xi) {
        const uint32_t x = (uint32_t)xi;
        if (B[x].empty()) continue;
        ++pivots;
        std::vector<Cand> C;
        for (size_t si = 0; si < B[x].size() && (int)C.size() < L_build; ++si) {
            const uint32_t *nout = knn.data() + (size_t)B[x][si] * nq_depth + 1;
            for (int r = 0; r < nq_depth - 1 && (int)C.size() < L_build; ++r) {
                const uint32_t c = nout[r];
                if (c == x || seen[c]) continue;
                seen[c] = 1;
                C.emplace_back(dist(X, d, x, c), c);
            }
        }
        for (auto &c : C) seen[c.second] = 0;
        std::sort(C.begin(), C.end(), cand_less);
        acquire(X, d, x, C, M, true, res);
        pj[x] = res;
        snap = res;
        for (uint32_t p : snap) reverse_update(X, d, pj, p, x, M, true, tmp);
    }
    int64_t pj_edges = 0;
    std::vector<uint32_t> rows((size_t)n * R, kNone);
    for (int64_t x = 0; x < n; ++x) {
        pj_edges += (int64_t)pj[x].size();
        std::copy(pj[x].begin(), pj[x].end(), rows.begin() + (size_t)x * R);
    }
    if (pj_dev) {
        std::vector<uint32_t> pr((size_t)n * M, kNone);
        for (int64_t x = 0; x < n; ++x) std::copy(pj[x].begin(), pj[x].end(), pr.begin() + (size_t)x * M);
        e = cudaMemcpyAsync(pj_dev, pr.data(), pr.size() * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "roar_build_index_literal: G_pj output");
    }

    // Enhancement: every row searched over the fixed G_pj (GPU), N'(x) by
    // Alg. 3 without fill over its result (GPU), in chunks.
    std::vector<std::vector<uint32_t>> gp = pj;   // G'
    {
        const int64_t CH = std::min<int64_t>(n, 65536);
        e = cudaMemcpyAsync(adj_dev, rows.data(), rows.size() * 4, cudaMemcpyHostToDevice, s);
        uint32_t *pid = nullptr, *xs = nullptr, *kept = nullptr;
        float *pd = nullptr;
        int32_t *nc = nullptr, *kc = nullptr;
        if (e == cudaSuccess) e = cudaMalloc(&pid, (size_t)CH * L_build * 4);
        if (e == cudaSuccess) e = cudaMalloc(&pd, (size_t)CH * L_build * 4);
        if (e == cudaSuccess) e = cudaMalloc(&xs, (size_t)CH * 4);
        if (e == cudaSuccess) e = cudaMalloc(&nc, (size_t)CH * 4);
        if (e == cudaSuccess) e = cudaMalloc(&kept, (size_t)CH * M * 4);
        if (e == cudaSuccess) e = cudaMalloc(&kc, (size_t)CH * 4);
        roar_index *gi = nullptr;
        if (e == cudaSuccess)
            rc = roar_index_create(n, d, X_dev, ROAR_F32, nullptr, nullptr, adj_dev, R, entry, 1u << 24, &gi);
        std::vector<uint32_t> hx((size_t)CH), hk((size_t)CH * M);
        std::vector<int32_t> hn((size_t)CH, L_build), hc((size_t)CH);
        std::vector<std::vector<uint32_t>> fwd((size_t)n);
        for (int64_t q0 = 0; e == cudaSuccess && rc == ROAR_OK && q0 < n; q0 += CH) {
            const int64_t qn = std::min(CH, n - q0);
            for (int64_t i = 0; i < qn; ++i) hx[i] = (uint32_t)(q0 + i);
            rc = roar_search(gi, X_dev + (size_t)q0 * d, qn, L_build, L_build, pid, pd, nullptr, nullptr, nullptr,
                             stream);
            if (rc != ROAR_OK) break;
            e = cudaMemcpyAsync(xs, hx.data(), (size_t)qn * 4, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(nc, hn.data(), (size_t)qn * 4, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) break;
            rc = roar_acquire(X_dev, n, d, xs, qn, pid, L_build, nc, M, 0, kept, kc, nullptr, stream);
            if (rc != ROAR_OK) break;
            e = cudaMemcpyAsync(hk.data(), kept, (size_t)qn * M * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), kc, (size_t)qn * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) break;
            for (int64_t i = 0; i < qn; ++i) {
                if (hc[i] < 0) {
                    set_error("roar_build_index_literal: a search returned an id outside the base set");
                    rc = ROAR_EINVAL;
                    break;
                }
                fwd[q0 + i].assign(hk.begin() + (size_t)i * M, hk.begin() + (size_t)i * M + hc[i]);
            }
        }
        roar_index_destroy(gi);
        cudaFree(pid);
        cudaFree(pd);
        cudaFree(xs);
        cudaFree(nc);
        cudaFree(kept);
        cudaFree(kc);
        if (e != cudaSuccess) return cuda_fail(e, "roar_build_index_literal: enhancement");
        if (rc != ROAR_OK) return rc;
        // In ascending x: G'(x) <- N'(x), then the reverse edges (no fill).
        for (int64_t xi = 0; xi < n; ++xi) {
            gp[xi] = fwd[xi];
            snap = fwd[xi];
            for (uint32_t p : snap) reverse_update(X, d, gp, p, (uint32_t)xi, M, false, tmp);
        }
    }

    // Final union: N_pj(x) followed by G'(x) minus N_pj(x).
    std::vector<int> deg((size_t)n, 0);
    std::fill(rows.begin(), rows.end(), kNone);
    for (int64_t x = 0; x < n; ++x) {
        uint32_t *r = rows.data() + (size_t)x * R;
        int k = 0;
        for (uint32_t u : pj[x]) r[k++] = u;
        for (uint32_t u : gp[x])
            if (std::find(pj[x].begin(), pj[x].end(), u) == pj[x].end() && k < R) r[k++] = u;
        deg[x] = k;
    }

    // Reachability repair (the rule in the header comment).
    int64_t repairs = 0, unreach0 = 0;
    {
        std::vector<unsigned char> reach((size_t)n);
        std::vector<uint32_t> queue((size_t)n);
        for (;;) {
            std::fill(reach.begin(), reach.end(), 0);
            int64_t head = 0, tail = 0;
            reach[entry] = 1;
            queue[tail++] = entry;
            while (head < tail) {
                const uint32_t v = queue[head++];
                for (int j = 0; j < deg[v]; ++j) {
                    const uint32_t w = rows[(size_t)v * R + j];
                    if (!reach[w]) {
                        reach[w] = 1;
                        queue[tail++] = w;
                    }
                }
            }
            if (repairs == 0) unreach0 = n - tail;
            if (tail == n) break;
            uint32_t u = 0;
            while (reach[u]) ++u;
            int64_t best = -1, bestfull = -1;
            float bd = INFINITY, bdf = INFINITY;
            for (int64_t r = 0; r < n; ++r) {
                if (!reach[r]) continue;
                const float dd = dist(X, d, u, (uint32_t)r);
                if (deg[r] < R) {
                    if (dd < bd) {
                        bd = dd;
                        best = r;
                    }
                } else if (dd < bdf) {
                    bdf = dd;
                    bestfull = r;
                }
            }
            if (best >= 0) rows[(size_t)best * R + deg[best]++] = u;
            else rows[(size_t)bestfull * R + R - 1] = u;
            ++repairs;
        }
    }
    e = cudaMemcpyAsync(adj_dev, rows.data(), rows.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "roar_build_index_literal: upload");
    int64_t fin = 0;
    for (int64_t x = 0; x < n; ++x) fin += deg[x];
    *entry_out = entry;
    if (stats) {
        double st[16] = {0};
        st[0] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_all).count();
        st[6] = (double)pivots;
        st[7] = (double)pj_edges;
        st[8] = (double)fin;
        st[9] = (double)unreach0;
        st[10] = (double)repairs;
        std::memcpy(stats, st, sizeof st);
    }
    return ROAR_OK;
}
