// RoarGraph index construction (Alg. 1-3, Sec. 4.2) for large inputs.
//
// The dense step (each training query's N_q nearest base rows) runs on the
// GPU through roar_knn. The rest runs in a batched form that is deterministic
// for any thread count:
//   projection:  every pivot's list N'(x) = AcquireNeighbors(x, C(x), M, fill)
//                is computed independently on host threads (Alg. 2, pivot
//                selection); then every node p receives the reverse edges
//                p -> x of all pivots x with p in N'(x) at once, re-pruned
//                with Alg. 3 (fill) when the list would exceed M (Alg. 2,
//                reverse-edge step);
//   enhancement: the rows are taken in chunks of doubling size; every row's
//                beam search runs on the GPU (roar_search) and its
//                supplementary list is AcquireNeighbors over the result and
//                the reverse edges it already has, without fill, on the GPU
//                (roar_acquire; Alg. 1, enhancement loop); then the chunk's
//                reverse edges are added the same batched way (their re-pruning
//                on the GPU too, hubs on host threads), and the next chunk
//                searches G_pj merged with all supplementary edges so far
//                (Alg. 1's final union, formed early): on data whose clusters
//                G_pj leaves unconnected, the reverse edges of the first rows
//                are what lets later searches leave the medoid's cluster;
//   repair:      any node the final graph cannot reach from the entry gets an
//                edge from the nearest reachable node the search finds.
// The sequential order of the paper's loops (each pivot seeing the reverse
// edges of earlier pivots) is replaced by these batched rounds, which is what
// makes the work parallel.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <utility>
#include <vector>

#include "roargraph.h"

namespace roar {
roar_status cuda_fail(cudaError_t e, const char *what);
void set_error(const char *msg);
}  // namespace roar

namespace {

using Cand = std::pair<float, uint32_t>;  // (distance, id)
constexpr uint32_t kNone = 0xFFFFFFFFu;

inline bool cand_less(const Cand &a, const Cand &b) {
    return a.first < b.first || (a.first == b.first && a.second < b.second);
}

// delta(a, b) = -<a, b>, FP32, 8 independent partial sums (vectorisable).
inline float neg_dot(const float *a, const float *b, int d) {
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int i = 0;
    for (; i + 8 <= d; i += 8)
        for (int j = 0; j < 8; ++j) s[j] += a[i + j] * b[i + j];
    float t = 0.0f;
    for (; i < d; ++i) t += a[i] * b[i];
    return -(((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])) + t);
}

template <class F>
void parallel_for(int64_t n, int threads, F &&f) {
    std::atomic<int64_t> next{0};
    const int64_t chunk = 256;
    auto work = [&](int tid) {
        for (;;) {
            const int64_t b = next.fetch_add(chunk);
            if (b >= n) break;
            const int64_t e = std::min(n, b + chunk);
            for (int64_t i = b; i < e; ++i) f(i, tid);
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto &th : pool) th.join();
}

// Alg. 3 over C sorted by (distance to x, id). Keeps the closest candidate,
// then every candidate closer to x than to each kept neighbour (strict), up
// to M; with fill, tops up to M from the remaining candidates in order.
int acquire(const float *X, int d, uint32_t x, const std::vector<Cand> &C, int M, bool fill,
            uint32_t *res) {
    int nr = 0;
    for (size_t i = 0; i < C.size() && nr < M; ++i) {
        const uint32_t c = C[i].second;
        if (c == x) continue;
        bool keep = true;
        for (int j = 0; j < nr && keep; ++j) {
            if (res[j] == c) keep = false;
            else if (!(C[i].first < neg_dot(X + (size_t)c * d, X + (size_t)res[j] * d, d))) keep = false;
        }
        if (nr == 0 || keep) res[nr++] = c;
    }
    if (fill) {
        for (size_t i = 0; i < C.size() && nr < M; ++i) {
            const uint32_t c = C[i].second;
            if (c == x) continue;
            bool dup = false;
            for (int j = 0; j < nr; ++j) dup |= res[j] == c;
            if (!dup) res[nr++] = c;
        }
    }
    return nr;
}

// Lists stored as [n][cap] with counts.
struct Lists {
    int64_t n = 0;
    int cap = 0;
    std::vector<uint32_t> v;
    std::vector<int> cnt;
    void init(int64_t n_, int cap_) {
        n = n_;
        cap = cap_;
        v.assign((size_t)n * cap, kNone);
        cnt.assign((size_t)n, 0);
    }
    uint32_t *row(int64_t i) { return v.data() + (size_t)i * cap; }
    const uint32_t *row(int64_t i) const { return v.data() + (size_t)i * cap; }
};

// GPU re-pruning for reverse-edge rounds without fill: a target whose list
// must be re-pruned and that received at most kGpuInc new edges in the round
// is batched through roar_acquire (FP32 fixed-order distances); busier
// targets (hubs) stay on the host.
constexpr int kGpuInc = 96;
struct GpuPrune {
    const float *X_dev = nullptr;
    int64_t n = 0;
    int d = 0, M = 0, CS = 0;
    int64_t rows = 0;  // batch capacity
    uint32_t *cand = nullptr, *out = nullptr, *srt = nullptr, *xs = nullptr;
    int32_t *nc = nullptr, *cnt = nullptr;
    std::vector<uint32_t> hcand, hout, hsrt, hxs;
    std::vector<int32_t> hnc, hcnt;
    void *stream = nullptr;
    cudaError_t init(const float *X, int64_t n_, int d_, int M_, int64_t rows_, void *stream_) {
        X_dev = X;
        n = n_;
        d = d_;
        M = M_;
        CS = M_ + kGpuInc;
        rows = rows_;
        stream = stream_;
        cudaError_t e = cudaMalloc(&cand, (size_t)rows * CS * 4);
        if (e == cudaSuccess) e = cudaMalloc(&srt, (size_t)rows * CS * 4);
        if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)rows * M * 4);
        if (e == cudaSuccess) e = cudaMalloc(&xs, (size_t)rows * 4);
        if (e == cudaSuccess) e = cudaMalloc(&nc, (size_t)rows * 4);
        if (e == cudaSuccess) e = cudaMalloc(&cnt, (size_t)rows * 4);
        if (e != cudaSuccess) return e;
        hcand.resize((size_t)rows * CS);
        hsrt.resize((size_t)rows * CS);
        hout.resize((size_t)rows * M);
        hxs.resize((size_t)rows);
        hnc.resize((size_t)rows);
        hcnt.resize((size_t)rows);
        return cudaSuccess;
    }
    ~GpuPrune() {
        cudaFree(cand);
        cudaFree(srt);
        cudaFree(out);
        cudaFree(xs);
        cudaFree(nc);
        cudaFree(cnt);
    }
};

// Batched reverse-edge round (Alg. 2 and Alg. 1's enhancement loop) for the
// forward edges of the sources x in [s0, s1): every node p gets p -> x for all
// such x with p in fwd(x); lists over M are re-pruned with Alg. 3. Without
// fill, the free slots left by the pruning are topped up with the remaining
// reverse edges, nearest first: the paper's sequential loop appends a reverse
// edge whenever the list has room, so its lists end up full of reverse edges
// after each pruning, and the top-up gives the batched round the same outcome.
// A node that many lists point to (a hub) keeps at most `max_in` of its
// reverse-edge candidates, the nearest ones, before pruning. Lists are
// updated in place; nodes without incoming edges keep theirs. Every changed
// node is flagged in `dirty` when it is given. With `gpu` (no fill only), the
// re-pruning of targets with at most kGpuInc new edges runs on the GPU.
roar_status add_reverse_edges(const float *X, int d, int M, bool fill, int threads, Lists &fwd, int max_in,
                              int64_t s0, int64_t s1, std::vector<unsigned char> *dirty = nullptr,
                              GpuPrune *gpu = nullptr) {
    const int64_t n = fwd.n;
    std::vector<int64_t> off((size_t)n + 1, 0);
    for (int64_t x = s0; x < s1; ++x)
        for (int j = 0; j < fwd.cnt[x]; ++j) ++off[fwd.row(x)[j] + 1];
    for (int64_t i = 0; i < n; ++i) off[i + 1] += off[i];
    std::vector<uint32_t> inc((size_t)off[n]);
    std::vector<int64_t> fillpos(off.begin(), off.end() - 1);
    for (int64_t x = s0; x < s1; ++x)  // ascending x: deterministic incoming order
        for (int j = 0; j < fwd.cnt[x]; ++j) inc[fillpos[fwd.row(x)[j]]++] = (uint32_t)x;
    fillpos.clear();
    fillpos.shrink_to_fit();
    std::vector<unsigned char> on_gpu(gpu && !fill ? (size_t)n : 0, 0);
    // own list first, then the incoming ids not in it (distinct, ascending)
    auto gather = [&](int64_t p, std::vector<uint32_t> &all) {
        const int nf = fwd.cnt[p];
        all.assign(fwd.row(p), fwd.row(p) + nf);
        for (int64_t k = off[p]; k < off[p + 1]; ++k) {
            const uint32_t x = inc[k];
            if (x == (uint32_t)p) continue;
            if (std::find(all.begin(), all.begin() + nf, x) == all.begin() + nf) all.push_back(x);
        }
    };
    parallel_for(n, threads, [&](int64_t p, int) {
        if (off[p] == off[p + 1]) return;
        if (dirty) (*dirty)[p] = 1;
        const int nf = fwd.cnt[p];
        std::vector<uint32_t> all;
        gather(p, all);
        const uint32_t *f = all.data();
        uint32_t *o = fwd.row(p);
        if ((int)all.size() <= M) {
            std::copy(all.begin(), all.end(), o);
            fwd.cnt[p] = (int)all.size();
            return;
        }
        if (!on_gpu.empty() && (int)all.size() - nf <= kGpuInc) {
            on_gpu[p] = 1;
            return;
        }
        std::vector<Cand> C;
        C.reserve(all.size());
        const float *pv = X + (size_t)p * d;
        for (uint32_t c : all) C.emplace_back(neg_dot(pv, X + (size_t)c * d, d), c);
        if ((int)C.size() > nf + max_in) {  // keep the own list and the nearest reverse edges
            std::vector<Cand> own(C.begin(), C.begin() + nf);
            std::nth_element(C.begin() + nf, C.begin() + nf + max_in, C.end(), cand_less);
            C.resize((size_t)(nf + max_in));
            std::copy(own.begin(), own.end(), C.begin());
        }
        std::sort(C.begin(), C.end(), cand_less);
        int r = acquire(X, d, (uint32_t)p, C, M, fill, o);
        if (!fill) {
            for (size_t i = 0; i < C.size() && r < M; ++i) {
                const uint32_t c = C[i].second;
                if (std::find(f, f + nf, c) != f + nf) continue;   // only reverse edges
                if (std::find(o, o + r, c) != o + r) continue;
                o[r++] = c;
            }
        }
        fwd.cnt[p] = r;
    });
    if (on_gpu.empty()) return ROAR_OK;
    std::vector<uint32_t> rows;
    for (int64_t p = 0; p < n; ++p)
        if (on_gpu[p]) rows.push_back((uint32_t)p);
    GpuPrune &g = *gpu;
    cudaStream_t s = (cudaStream_t)g.stream;
    for (size_t b0 = 0; b0 < rows.size(); b0 += (size_t)g.rows) {
        const int64_t nb = (int64_t)std::min(rows.size() - b0, (size_t)g.rows);
        parallel_for(nb, threads, [&](int64_t i, int) {
            const int64_t p = rows[b0 + i];
            std::vector<uint32_t> all;
            gather(p, all);
            uint32_t *r = g.hcand.data() + (size_t)i * g.CS;
            std::copy(all.begin(), all.end(), r);
            std::fill(r + all.size(), r + g.CS, kNone);
            g.hxs[i] = (uint32_t)p;
            g.hnc[i] = (int32_t)all.size();
        });
        cudaError_t e = cudaMemcpyAsync(g.cand, g.hcand.data(), (size_t)nb * g.CS * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.xs, g.hxs.data(), (size_t)nb * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.nc, g.hnc.data(), (size_t)nb * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return roar::cuda_fail(e, "roar_build_index: reverse-edge upload");
        roar_status rc = roar_acquire(g.X_dev, g.n, g.d, g.xs, nb, g.cand, g.CS, g.nc, M, 0, g.out, g.cnt, g.srt,
                                      g.stream);
        if (rc != ROAR_OK) return rc;
        e = cudaMemcpyAsync(g.hout.data(), g.out, (size_t)nb * M * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.hsrt.data(), g.srt, (size_t)nb * g.CS * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.hcnt.data(), g.cnt, (size_t)nb * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return roar::cuda_fail(e, "roar_build_index: reverse-edge prune");
        std::atomic<bool> bad{false};
        parallel_for(nb, threads, [&](int64_t i, int) {
            const int64_t p = rows[b0 + i];
            const uint32_t *f = g.hcand.data() + (size_t)i * g.CS;   // own list: the first nf ids
            const int nf = fwd.cnt[p];
            const uint32_t *srt = g.hsrt.data() + (size_t)i * g.CS;
            const int r0 = g.hcnt[i];
            if (r0 < 0) {
                bad = true;
                return;
            }
            uint32_t *o = fwd.row(p);
            std::copy(g.hout.data() + (size_t)i * M, g.hout.data() + (size_t)i * M + r0, o);
            int r = r0;
            for (int j = 0; j < g.CS && r < M && srt[j] != kNone; ++j) {   // top-up: reverse edges, nearest first
                const uint32_t c = srt[j];
                if (c == (uint32_t)p) continue;
                if (std::find(f, f + nf, c) != f + nf) continue;
                if (std::find(o, o + r, c) != o + r) continue;
                o[r++] = c;
            }
            fwd.cnt[p] = r;
        });
        if (bad) {
            roar::set_error("roar_build_index: an edge points outside the base set");
            return ROAR_EINVAL;
        }
    }
    return ROAR_OK;
}

// Row x of the searched / final graph: N_pj(x) followed by the supplementary
// edges not already in it (Alg. 1's final union); returns the row's length.
int merge_row(const Lists &pj, const Lists &ce, int64_t x, uint32_t *row, int R) {
    int k = 0;
    for (int j = 0; j < pj.cnt[x]; ++j) row[k++] = pj.row(x)[j];
    for (int j = 0; j < ce.cnt[x]; ++j) {
        const uint32_t u = ce.row(x)[j];
        bool dup = false;
        for (int t = 0; t < pj.cnt[x]; ++t) dup |= pj.row(x)[t] == u;
        if (!dup) row[k++] = u;
    }
    for (int j = k; j < R; ++j) row[j] = kNone;
    return k;
}

// Page-locks an existing host buffer for the lifetime of the guard (faster
// repeated uploads); if the driver refuses, the buffer stays pageable.
struct HostPin {
    void *p = nullptr;
    HostPin(void *ptr, size_t bytes) {
        if (cudaHostRegister(ptr, bytes, cudaHostRegisterDefault) == cudaSuccess) p = ptr;
        else cudaGetLastError();
    }
    ~HostPin() {
        if (p) cudaHostUnregister(p);
    }
    HostPin(const HostPin &) = delete;
    HostPin &operator=(const HostPin &) = delete;
};

double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Progress lines on stderr when ROAR_BUILD_LOG is set (long builds).
void build_log(const char *fmt, double a = 0, double b = 0, double c = 0) {
    static const bool on = std::getenv("ROAR_BUILD_LOG") != nullptr;
    if (!on) return;
    std::fprintf(stderr, "[roar_build] ");
    std::fprintf(stderr, fmt, a, b, c);
    std::fprintf(stderr, "\n");
    std::fflush(stderr);
}

// BFS from entry over [n][R] adjacency; returns unreachable ids ascending.
std::vector<uint32_t> unreachable(const std::vector<uint32_t> &adj, int64_t n, int R, uint32_t entry) {
    std::vector<unsigned char> seen((size_t)n, 0);
    std::vector<uint32_t> q;
    q.reserve((size_t)n);
    q.push_back(entry);
    seen[entry] = 1;
    for (size_t h = 0; h < q.size(); ++h) {
        const uint32_t *row = adj.data() + (size_t)q[h] * R;
        for (int j = 0; j < R; ++j) {
            const uint32_t u = row[j];
            if (u == kNone) continue;
            if (!seen[u]) {
                seen[u] = 1;
                q.push_back(u);
            }
        }
    }
    std::vector<uint32_t> out;
    for (int64_t i = 0; i < n; ++i)
        if (!seen[i]) out.push_back((uint32_t)i);
    return out;
}

}  // namespace

using namespace roar;

extern "C" roar_status roar_medoid(const float *X_host, int64_t n, int32_t d, int32_t threads,
                                   uint32_t *entry) {
    if (!X_host || n < 1 || d < 1 || !entry) return ROAR_EINVAL;
    if (threads < 1) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    // FP64 mean with fixed per-chunk partial sums (deterministic for any thread count).
    const int64_t chunk = 65536;
    const int64_t nch = (n + chunk - 1) / chunk;
    std::vector<double> part((size_t)nch * d, 0.0);
    parallel_for(nch, threads, [&](int64_t c, int) {
        double *p = part.data() + (size_t)c * d;
        for (int64_t i = c * chunk; i < std::min(n, (c + 1) * chunk); ++i)
            for (int j = 0; j < d; ++j) p[j] += (double)X_host[(size_t)i * d + j];
    });
    std::vector<double> mu((size_t)d, 0.0);
    for (int64_t c = 0; c < nch; ++c)
        for (int j = 0; j < d; ++j) mu[j] += part[(size_t)c * d + j];
    for (int j = 0; j < d; ++j) mu[j] /= (double)n;
    std::vector<double> bestd((size_t)nch, INFINITY);
    std::vector<int64_t> besti((size_t)nch, -1);
    parallel_for(nch, threads, [&](int64_t c, int) {
        for (int64_t i = c * chunk; i < std::min(n, (c + 1) * chunk); ++i) {
            double s = 0.0;
            for (int j = 0; j < d; ++j) {
                const double t = (double)X_host[(size_t)i * d + j] - mu[j];
                s += t * t;
            }
            if (s < bestd[c]) {
                bestd[c] = s;
                besti[c] = i;
            }
        }
    });
    int64_t b = besti[0];
    double bd = bestd[0];
    for (int64_t c = 1; c < nch; ++c)
        if (bestd[c] < bd) {
            bd = bestd[c];
            b = besti[c];
        }
    *entry = (uint32_t)b;
    return ROAR_OK;
}

extern "C" roar_status roar_build_index(const float *X_dev, int64_t n, int32_t d, const float *T_dev,
                                        int64_t nt, int32_t nq_depth, int32_t M, int32_t L_build,
                                        int32_t threads, uint32_t *adj_dev, uint32_t *pj_dev, uint32_t *entry_out,
                                        double *stats, void *stream) {
    if (!X_dev || !T_dev || !adj_dev || !entry_out || n < 2 || nt < 1 || d < 4 || d % 4 ||
        d > 1024 || nq_depth < 2 || nq_depth > 128 || nq_depth > n || M < 1 || 2 * M > ROAR_MAX_RMAX ||
        L_build < M || L_build > ROAR_MAX_L) {
        set_error("roar_build_index: bad arguments");
        return ROAR_EINVAL;
    }
    if (threads < 1) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    cudaStream_t s = (cudaStream_t)stream;
    const auto t_all = std::chrono::steady_clock::now();
    double st[16] = {0};
    roar_status rc = ROAR_OK;
    const int R = 2 * M;

    // Base rows on the host for the pruning distances.
    std::vector<float> X((size_t)n * d);
    cudaError_t e = cudaMemcpyAsync(X.data(), X_dev, X.size() * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "roar_build_index: copy X");

    uint32_t entry = 0;
    roar_medoid(X.data(), n, d, threads, &entry);

    // Alg. 1 input: N_q nearest base rows of every training query (GPU).
    auto t0 = std::chrono::steady_clock::now();
    std::vector<uint32_t> knn((size_t)nt * nq_depth);
    {
        uint32_t *ki = nullptr;
        float *kd = nullptr;
        e = cudaMalloc(&ki, knn.size() * 4);
        if (e == cudaSuccess) e = cudaMalloc(&kd, knn.size() * 4);
        if (e != cudaSuccess) {
            cudaFree(ki);
            cudaGetLastError();
            return ROAR_ENOMEM;
        }
        rc = roar_knn(T_dev, nt, X_dev, n, d, nq_depth, ki, kd, stream);
        if (rc == ROAR_OK) {
            e = cudaMemcpyAsync(knn.data(), ki, knn.size() * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = cuda_fail(e, "roar_build_index: copy kNN");
        }
        cudaFree(ki);
        cudaFree(kd);
        if (rc != ROAR_OK) return rc;
    }
    st[1] = seconds_since(t0);
    build_log("kNN of %.0f training queries done in %.1f s", (double)nt, st[1]);

    // Alg. 1, bipartite step: base node x = 1-NN(t) gets the edge x -> t.
    t0 = std::chrono::steady_clock::now();
    std::vector<int64_t> boff((size_t)n + 1, 0);
    for (int64_t t = 0; t < nt; ++t) ++boff[knn[(size_t)t * nq_depth] + 1];
    for (int64_t i = 0; i < n; ++i) boff[i + 1] += boff[i];
    std::vector<uint32_t> bq((size_t)nt);
    {
        std::vector<int64_t> pos(boff.begin(), boff.end() - 1);
        for (int64_t t = 0; t < nt; ++t) bq[pos[knn[(size_t)t * nq_depth]]++] = (uint32_t)t;
    }
    // Alg. 2, pivot selection: each pivot selects from its bridges' other neighbours.
    Lists pj;
    pj.init(n, M);
    std::atomic<int64_t> pivots{0};
    std::vector<std::vector<unsigned char>> seen_t((size_t)threads);
    parallel_for(n, threads, [&](int64_t x, int tid) {
        if (boff[x] == boff[x + 1]) return;
        ++pivots;
        auto &seen = seen_t[tid];
        if (seen.empty()) seen.assign((size_t)n, 0);
        std::vector<Cand> C;
        C.reserve((size_t)L_build);
        const float *xv = X.data() + (size_t)x * d;
        for (int64_t b = boff[x]; b < boff[x + 1] && (int)C.size() < L_build; ++b) {
            const uint32_t *nout = knn.data() + (size_t)bq[b] * nq_depth + 1;
            for (int r = 0; r < nq_depth - 1 && (int)C.size() < L_build; ++r) {
                const uint32_t c = nout[r];
                if (c == (uint32_t)x || c == kNone || seen[c]) continue;
                seen[c] = 1;
                C.emplace_back(neg_dot(xv, X.data() + (size_t)c * d, d), c);
            }
        }
        for (auto &c : C) seen[c.second] = 0;
        std::sort(C.begin(), C.end(), cand_less);
        pj.cnt[x] = acquire(X.data(), d, (uint32_t)x, C, M, true, pj.row(x));
    });
    // Alg. 2, reverse-edge step, batched.
    if ((rc = add_reverse_edges(X.data(), d, M, true, threads, pj, 4 * L_build, 0, n)) != ROAR_OK) return rc;
    // The enhancement searches start at the medoid and walk G_pj: a medoid
    // that no pivot selected has no edges there and every search would stop
    // at once. Such a medoid gets a list as a pivot would, from its own
    // nearest base rows (exact kNN on the GPU), with Alg. 3 and fill.
    if (pj.cnt[entry] == 0) {
        uint32_t *ki = nullptr;
        float *kd = nullptr;
        const int kk = std::min<int64_t>(std::min(128, L_build), n);
        e = cudaMalloc(&ki, (size_t)kk * 4);
        if (e == cudaSuccess) e = cudaMalloc(&kd, (size_t)kk * 4);
        std::vector<uint32_t> hid((size_t)kk);
        std::vector<float> hd((size_t)kk);
        if (e == cudaSuccess) rc = roar_knn(X_dev + (size_t)entry * d, 1, X_dev, n, d, kk, ki, kd, stream);
        if (e == cudaSuccess && rc == ROAR_OK) {
            e = cudaMemcpy(hid.data(), ki, (size_t)kk * 4, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(hd.data(), kd, (size_t)kk * 4, cudaMemcpyDeviceToHost);
        }
        cudaFree(ki);
        cudaFree(kd);
        if (e != cudaSuccess) return cuda_fail(e, "roar_build_index: medoid list");
        if (rc != ROAR_OK) return rc;
        std::vector<Cand> C;
        for (int j = 0; j < kk; ++j)
            if (hid[j] != entry && hid[j] != kNone) C.emplace_back(hd[j], hid[j]);
        pj.cnt[entry] = acquire(X.data(), d, entry, C, M, true, pj.row(entry));
        build_log("medoid had no projected edges: gave it %.0f", (double)pj.cnt[entry]);
    }
    st[2] = seconds_since(t0);
    build_log("projection done in %.1f s (%.0f pivots)", st[2], (double)pivots.load());
    int64_t pj_edges = 0;
    for (int64_t i = 0; i < n; ++i) pj_edges += pj.cnt[i];
    if (pj_dev) {  // G_pj as it stands before enhancement
        std::vector<uint32_t> pjrows((size_t)n * M, kNone);
        parallel_for(n, threads, [&](int64_t x, int) {
            std::copy(pj.row(x), pj.row(x) + pj.cnt[x], pjrows.data() + (size_t)x * M);
        });
        e = cudaMemcpyAsync(pj_dev, pjrows.data(), pjrows.size() * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "roar_build_index: G_pj output");
    }

    // Alg. 1, enhancement loop: beam search of every base row (GPU), AcquireNeighbors
    // without fill, reverse edges. The rows are processed in chunks of
    // doubling size (1024, 1024, 2048, ... up to n / 32, at least 131072 and
    // at most 524288), and each chunk
    // searches G_pj merged with the supplementary edges of the chunks before
    // it: a reverse edge p -> x added for an earlier row gives later searches
    // a route from the medoid's region to x's, which G_pj alone may lack (on
    // well separated clusters it has no edge between them). A row's own list
    // is pruned from its search result together with the reverse edges it has
    // already received.
    t0 = std::chrono::steady_clock::now();
    Lists ce;
    ce.init(n, M);
    std::vector<uint32_t> adj((size_t)n * R, kNone);
    HostPin adj_pin(adj.data(), adj.size() * 4);      // uploaded once per chunk
    std::vector<int> deg((size_t)n, 0);
    std::vector<unsigned char> dirty((size_t)n, 1);  // rows whose merged form is stale
    double t_merge = 0, t_search = 0, t_prune = 0, t_rev = 0;
    {
        // Per chunk: search results (L_build ids) and the reverse edges each row
        // has received (M ids) form that row's candidates for roar_acquire.
        const int CS = L_build + M;
        uint32_t *pid = nullptr, *cand = nullptr, *kept = nullptr, *xs = nullptr;
        int32_t *ncand = nullptr, *kcnt = nullptr;
        float *pdist = nullptr;
        const int64_t max_chunk = std::min<int64_t>(n, std::min<int64_t>(524288, std::max<int64_t>(131072, n / 32)));
        e = cudaMalloc(&pid, (size_t)max_chunk * L_build * 4);
        if (e == cudaSuccess) e = cudaMalloc(&pdist, (size_t)max_chunk * L_build * 4);
        if (e == cudaSuccess) e = cudaMalloc(&cand, (size_t)max_chunk * CS * 4);
        if (e == cudaSuccess) e = cudaMalloc(&kept, (size_t)max_chunk * M * 4);
        if (e == cudaSuccess) e = cudaMalloc(&xs, (size_t)max_chunk * 4);
        if (e == cudaSuccess) e = cudaMalloc(&ncand, (size_t)max_chunk * 4);
        if (e == cudaSuccess) e = cudaMalloc(&kcnt, (size_t)max_chunk * 4);
        std::vector<uint32_t> hxs((size_t)max_chunk);
        std::vector<int32_t> hk((size_t)max_chunk);
        if (e == cudaSuccess) {
            std::vector<int32_t> nc((size_t)max_chunk, CS);
            e = cudaMemcpyAsync(ncand, nc.data(), nc.size() * 4, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        GpuPrune gprune;
        if (e == cudaSuccess) e = gprune.init(X_dev, n, d, M, std::min<int64_t>(n, 262144), stream);
        roar_index *gi = nullptr;
        if (e == cudaSuccess)
            rc = roar_index_create(n, d, X_dev, ROAR_F32, nullptr, nullptr, adj_dev, R, entry, 32768, &gi);
        int64_t q0 = 0;
        while (e == cudaSuccess && rc == ROAR_OK && q0 < n) {
            const int64_t qn = std::min(n - q0, std::min(max_chunk, std::max<int64_t>(1024, q0)));
            auto tp = std::chrono::steady_clock::now();
            parallel_for(n, threads, [&](int64_t x, int) {
                if (!dirty[x]) return;
                dirty[x] = 0;
                deg[x] = merge_row(pj, ce, x, adj.data() + (size_t)x * R, R);
            });
            e = cudaMemcpyAsync(adj_dev, adj.data(), adj.size() * 4, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) break;
            t_merge += seconds_since(tp);
            tp = std::chrono::steady_clock::now();
            rc = roar_search(gi, X_dev + (size_t)q0 * d, qn, L_build, L_build, pid, pdist, nullptr,
                             nullptr, nullptr, stream);
            if (rc != ROAR_OK) break;
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) break;
            t_search += seconds_since(tp);
            tp = std::chrono::steady_clock::now();
            // Candidate rows: [search results | received reverse edges, padded].
            parallel_for(qn, threads, [&](int64_t i, int) {
                const int64_t x = q0 + i;
                uint32_t *r = ce.row(x);
                for (int j = ce.cnt[x]; j < M; ++j) r[j] = kNone;
                hxs[i] = (uint32_t)x;
            });
            e = cudaMemcpy2DAsync(cand, (size_t)CS * 4, pid, (size_t)L_build * 4, (size_t)L_build * 4, (size_t)qn,
                                  cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(cand + L_build, (size_t)CS * 4, ce.row(q0), (size_t)M * 4, (size_t)M * 4,
                                      (size_t)qn, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(xs, hxs.data(), (size_t)qn * 4, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) break;
            rc = roar_acquire(X_dev, n, d, xs, qn, cand, CS, ncand, M, 0, kept, kcnt, nullptr, stream);
            if (rc != ROAR_OK) break;
            e = cudaMemcpyAsync(ce.row(q0), kept, (size_t)qn * M * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hk.data(), kcnt, (size_t)qn * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) break;
            bool bad = false;
            for (int64_t i = 0; i < qn; ++i) {
                bad |= hk[i] < 0;
                ce.cnt[q0 + i] = hk[i] < 0 ? 0 : hk[i];
                dirty[q0 + i] = 1;
            }
            if (bad) {
                set_error("roar_build_index: a search returned an id outside the base set");
                rc = ROAR_EINVAL;
                break;
            }
            t_prune += seconds_since(tp);
            tp = std::chrono::steady_clock::now();
            rc = add_reverse_edges(X.data(), d, M, false, threads, ce, 4 * L_build, q0, q0 + qn, &dirty, &gprune);
            if (rc != ROAR_OK) break;
            t_rev += seconds_since(tp);
            q0 += qn;
            build_log("enhancement: searched %.0f of %.0f rows (%.1f s)", (double)q0, (double)n,
                      seconds_since(t0));
        }
        roar_index_destroy(gi);
        cudaFree(pid);
        cudaFree(pdist);
        cudaFree(cand);
        cudaFree(kept);
        cudaFree(xs);
        cudaFree(ncand);
        cudaFree(kcnt);
        if (e != cudaSuccess) return cuda_fail(e, "roar_build_index: enhancement search");
        if (rc != ROAR_OK) return rc;
    }
    st[3] = seconds_since(t0);
    // Alg. 1, final union: N_pj followed by the new edges.
    t0 = std::chrono::steady_clock::now();
    parallel_for(n, threads, [&](int64_t x, int) {
        if (dirty[x]) deg[x] = merge_row(pj, ce, x, adj.data() + (size_t)x * R, R);
    });
    st[4] = seconds_since(t0);
    build_log("enhancement done: search+prune %.1f s, merge %.1f s", st[3], st[4]);
    build_log("enhancement split: merge+upload %.1f s, GPU search %.1f s, prune %.1f s", t_merge, t_search, t_prune);
    build_log("enhancement split: reverse edges %.1f s", t_rev);

    // Reachability repair: each unreachable node gets an edge from the
    // nearest node (among the 16 the search finds from the entry) that still
    // has a free slot; repeated until every node is reachable.
    t0 = std::chrono::steady_clock::now();
    int64_t repairs = 0, unreach0 = -1, unreach_final = 0;
    {
        constexpr int KR = 16;
        for (int round = 0; round < 32; ++round) {
            std::vector<uint32_t> U = unreachable(adj, n, R, entry);
            if (unreach0 < 0) unreach0 = (int64_t)U.size();
            unreach_final = (int64_t)U.size();
            build_log("repair round %.0f: %.0f unreachable (%.1f s)", (double)round, (double)U.size(),
                      seconds_since(t0));
            if (U.empty()) break;
            if (round >= 3) {
                // Rare leftovers whose nearby nodes are all full: link each from
                // any reachable node with a free slot.
                std::vector<unsigned char> isU((size_t)n, 0);
                for (uint32_t u : U) isU[u] = 1;
                int64_t cur = 0;
                for (uint32_t u : U) {
                    while (cur < n && (isU[cur] || deg[cur] >= R)) ++cur;
                    if (cur >= n) break;
                    adj[(size_t)cur * R + deg[cur]++] = u;
                    ++repairs;
                }
                continue;
            }
            e = cudaMemcpyAsync(adj_dev, adj.data(), adj.size() * 4, cudaMemcpyHostToDevice, s);
            std::vector<float> Q(U.size() * (size_t)d);
            for (size_t i = 0; i < U.size(); ++i)
                std::memcpy(&Q[i * d], X.data() + (size_t)U[i] * d, (size_t)d * 4);
            float *qd = nullptr, *od = nullptr;
            uint32_t *oi = nullptr;
            if (e == cudaSuccess) e = cudaMalloc(&qd, Q.size() * 4);
            if (e == cudaSuccess) e = cudaMalloc(&oi, U.size() * KR * 4);
            if (e == cudaSuccess) e = cudaMalloc(&od, U.size() * KR * 4);
            if (e == cudaSuccess) e = cudaMemcpyAsync(qd, Q.data(), Q.size() * 4, cudaMemcpyHostToDevice, s);
            roar_index *gi = nullptr;
            if (e == cudaSuccess)
                rc = roar_index_create(n, d, X_dev, ROAR_F32, nullptr, nullptr, adj_dev, R, entry, 32768, &gi);
            if (e == cudaSuccess && rc == ROAR_OK)
                rc = roar_search(gi, qd, (int64_t)U.size(), KR, 64, oi, od, nullptr, nullptr, nullptr, stream);
            std::vector<uint32_t> r(U.size() * KR, kNone);
            if (e == cudaSuccess && rc == ROAR_OK)
                e = cudaMemcpyAsync(r.data(), oi, r.size() * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            roar_index_destroy(gi);
            cudaFree(qd);
            cudaFree(oi);
            cudaFree(od);
            if (e != cudaSuccess) return cuda_fail(e, "roar_build_index: repair");
            if (rc != ROAR_OK) return rc;
            int64_t added = 0;
            for (size_t i = 0; i < U.size(); ++i) {
                for (int j = 0; j < KR; ++j) {
                    const uint32_t src = r[i * KR + j];
                    if (src == kNone || deg[src] >= R) continue;
                    uint32_t *row = adj.data() + (size_t)src * R;
                    bool dup = false;
                    for (int t = 0; t < deg[src]; ++t) dup |= row[t] == U[i];
                    if (!dup) {
                        row[deg[src]++] = U[i];
                        ++added;
                    }
                    break;
                }
            }
            repairs += added;
            if (added == 0) break;
        }
    }
    st[5] = seconds_since(t0);
    e = cudaMemcpyAsync(adj_dev, adj.data(), adj.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "roar_build_index: upload");
    int64_t fin_edges = 0;
    for (int64_t i = 0; i < n; ++i) fin_edges += deg[i];
    *entry_out = entry;
    st[0] = seconds_since(t_all);
    st[6] = (double)pivots.load();
    st[7] = (double)pj_edges;
    st[8] = (double)fin_edges;
    st[9] = (double)unreach0;
    st[10] = (double)repairs;
    st[11] = (double)unreach_final;
    if (stats) std::memcpy(stats, st, sizeof st);
    return ROAR_OK;
}
