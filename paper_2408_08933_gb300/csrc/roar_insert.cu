// Insertion through the saved bipartite graph (Sec. 5.7): new base rows join
// a built RoarGraph without a rebuild. The result is that of inserting rows
// n_old .. n_total-1 one at a time in id order, where for row v:
//   1. beam search of X[v] over the current graph (width L, the whole pool);
//   2. the first pool entry b that some training query is connected to (b in
//      N_out(t), or b is t's nearest base row, its pivot);
//   3. q = the connected query nearest to v (FP32 fixed-order dot, ties by id);
//   4. N(v) = AcquireNeighbors with fill over N_out(q) (Alg. 3, roar_acquire,
//      which sorts by (delta(v, c), id)); with no connected pool entry, over
//      the search pool;
//   5. v's row is N(v); each p in N(v) gets p -> v, appended when p's row has
//      room, else p's row and v are re-pruned to R with fill;
//   6. v joins N_out(q) while it has room.
// Every keep / drop decision is FP32 with the search's fixed summation order.
//
// The work is done in windows of W rows, speculatively, with the same result:
//   - the searches of every window row without a usable result run in one
//     launch on the graph as it stands, each recording the nodes it expands
//     (the only adjacency rows a search reads);
//   - N(v) for every window row comes from one batched roar_acquire;
//   - rows are then applied in order on the host copy of the graph. Each
//     graph row carries the sequence number of the last insertion that
//     changed it; a search is still exact if no row it expanded changed after
//     it ran, since a beam search is a function of the rows it expands, or if
//     the only changes are new neighbours appended to such rows that would not
//     have entered the pool: each one's distance to the query is above the
//     pool's L-th distance when the row was expanded (recorded by the search),
//     so it would only have counted as a visit (the visits stay below the
//     cap). The first row whose search fails this test ends the window's apply; its
//     search is redone in the next window (on the graph with every earlier
//     row applied, hence exact), and later rows keep theirs while they pass.
//     A list N(v) is redone when N_out(q) grew since it was computed;
//   - re-prunes of full rows are batched, and flushed before a row with one
//     pending is read again;
//   - the rows changed by the window are scattered to the device graph in one
//     kernel before the next window's searches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "roar_internal.cuh"

namespace roar {
roar_status cuda_fail(cudaError_t e, const char *what);
void set_error(const char *msg);
}  // namespace roar

using namespace roar;

namespace {

using Clock = std::chrono::steady_clock;
double since(Clock::time_point t0) { return std::chrono::duration<double>(Clock::now() - t0).count(); }

constexpr uint32_t kMaxVisits = 16384u;   // the insertion searches' visit cap

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

// (dist, id) total order of the search.
__device__ __forceinline__ bool less_entry(float da, uint32_t ia, float db, uint32_t ib) {
    return da < db || (da == db && ia < ib);
}

// Steps 2-3 on the device: for row r, the query t in cids[coff[r] ..
// coff[r + 1]) nearest to X[xs[r]], by (delta, id) with delta = -<x, T[t]> in
// the search's fixed FP32 order (element i accumulates, fmaf in increasing i,
// into lane (i >> 2) & 31 of 32 partial sums from +0, then the butterfly
// s_l + s_(l xor o) for o = 16, 8, 4, 2, 1). One 256-thread block per row,
// a warp per candidate; the minimum of a total order does not depend on
// which warp saw which candidate.
__global__ void __launch_bounds__(256) nearest_query(const float *__restrict__ X, const float *__restrict__ T,
                                                     int d, const uint32_t *__restrict__ xs,
                                                     const int64_t *__restrict__ coff,
                                                     const uint32_t *__restrict__ cids, uint32_t *__restrict__ best) {
    __shared__ float sd[8];
    __shared__ uint32_t si[8];
    const int r = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int d4 = d >> 2;
    const float4 *x4 = reinterpret_cast<const float4 *>(X + (size_t)xs[r] * d);
    float bd = 0.0f;
    uint32_t bi = 0xFFFFFFFFu;
    for (int64_t j = coff[r] + warp; j < coff[r + 1]; j += 8) {
        const uint32_t t = cids[j];
        const float4 *t4 = reinterpret_cast<const float4 *>(T + (size_t)t * d);
        float acc = 0.0f;
        for (int ch = lane; ch < d4; ch += 32) {
            const float4 a = __ldg(x4 + ch), b = __ldg(t4 + ch);
            acc = fmaf(a.x, b.x, acc);
            acc = fmaf(a.y, b.y, acc);
            acc = fmaf(a.z, b.z, acc);
            acc = fmaf(a.w, b.w, acc);
        }
        for (int o = 16; o >= 1; o >>= 1) acc = acc + __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        const float dt = -acc;
        if (bi == 0xFFFFFFFFu || less_entry(dt, t, bd, bi)) {
            bd = dt;
            bi = t;
        }
    }
    if (lane == 0) {
        sd[warp] = bd;
        si[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w)
            if (si[w] != 0xFFFFFFFFu && (bi == 0xFFFFFFFFu || less_entry(sd[w], si[w], bd, bi))) {
                bd = sd[w];
                bi = si[w];
            }
        best[r] = bi;
    }
}

// Row i of rows[m][R] becomes graph row dst[i].
__global__ void scatter_rows(uint32_t *__restrict__ adj, int R, const uint32_t *__restrict__ rows,
                             const int64_t *__restrict__ dst, int64_t m) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m * R) return;
    adj[dst[i / R] * R + i % R] = rows[i];
}

template <class T>
cudaError_t dalloc(T **p, size_t count) {
    return cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T));
}

struct Inserter {
    // inputs
    const float *X_dev;
    int64_t n_total, n_old;
    int d, R, M, L, W;
    const float *T;
    int32_t nout_cap;
    uint32_t *nout;
    int32_t *nout_cnt;
    int32_t *chosen_q;
    uint32_t *adj_dev;
    int64_t nt;
    uint32_t entry;
    cudaStream_t s;
    roar_index *gi = nullptr;
    // host graph and bookkeeping
    std::vector<uint32_t> adj;
    std::vector<float> Xnew;
    // Queries connected to each base row: the input's (CSR, a query may be
    // listed twice for one row, which does not change a nearest-query pick),
    // then those added for the inserted rows.
    std::vector<int64_t> inc_off;
    std::vector<uint32_t> inc_ids;
    std::vector<std::vector<uint32_t>> inc_new;
    std::vector<int64_t> stamp;               // last insertion (sequence number) that changed the row
    std::vector<int64_t> rewrite;             // last insertion that rewrote it (set or re-pruned)
    std::vector<int32_t> pos_seq;             // [n_total][R]: the insertion that appended the entry there
    std::vector<char> pend_mark, chg_mark;
    int64_t applied = 0;                      // rows inserted so far
    // window slots (row v lives in slot v % W)
    int TC = 0, CS = 0;
    std::vector<int64_t> sl_v, sl_snap, sl_q;
    std::vector<uint32_t> sl_hops, sl_pool, sl_trace, sl_acq, sl_vis;
    std::vector<float> sl_bound;
    std::vector<int32_t> sl_st;
    std::vector<int32_t> sl_acq_n, sl_acq_from;
    std::vector<char> sl_acq_ok;
    // pending re-prunes and changed rows
    std::vector<int64_t> pend, chg;
    // device buffers
    float *dq = nullptr, *ddist = nullptr;
    uint32_t *dids = nullptr, *dhops = nullptr, *dtrace = nullptr, *dvis = nullptr;
    float *dbound = nullptr;
    int32_t *dst = nullptr;
    uint32_t *dxs = nullptr, *dcand = nullptr, *dout = nullptr, *drows = nullptr;
    int32_t *dnc = nullptr, *dcnt = nullptr;
    int64_t *ddst = nullptr;
    float *dT = nullptr;                       // training queries on the device
    uint32_t *dcids = nullptr, *dxs_pick = nullptr, *dbest = nullptr;
    int64_t *dcoff = nullptr;
    int64_t cids_cap = 0;
    std::vector<uint32_t> hxs_pick, hbest;
    int64_t acq_cap = 0, chg_cap = 0;
    // host staging
    std::vector<float> hq;
    std::vector<uint32_t> hbuf, hxs, hout;
    std::vector<int32_t> hnc, hcnt;
    std::vector<int64_t> hdst;
    // windows, searches, lists, lists redone, re-prune batches, rows re-pruned;
    // seconds in: setup, searches, lists, applying (re-prunes included),
    // re-prunes, scatters, query picks; windows whose apply stopped at a
    // search that expanded rewritten rows, or only rows appended to
    static constexpr int kStats = 15;
    double stats[kStats] = {};

    roar_status fail(cudaError_t e, const char *what) { return cuda_fail(e, what); }

    bool usable(int slot) const {
        const int64_t snap = sl_snap[slot];
        if (snap < 0) return false;
        if (snap == applied) return true;
        if (sl_hops[slot] > (uint32_t)TC) return false;
        const uint32_t *tr = sl_trace.data() + (size_t)slot * TC;
        const float *bd = sl_bound.data() + (size_t)slot * TC;
        const float *xu = Xnew.data() + (size_t)(sl_v[slot] - n_old) * d;
        constexpr int kSeen = 64;
        uint32_t seen[kSeen];
        int nseen = 0;
        for (uint32_t i = 0; i < sl_hops[slot]; ++i) {
            const uint32_t e = tr[i];
            if (stamp[e] < snap) continue;
            if (rewrite[e] >= snap) return false;
            // Only appended to since the search: each new neighbour must stay
            // out of the pool (distance above the bound), ties are refused.
            for (int j = 0; j < R; ++j) {
                if (pos_seq[(size_t)e * R + j] < snap) continue;
                const uint32_t v = adj[(size_t)e * R + j];
                const float dv = -dot_fixed_host(xu, Xnew.data() + (size_t)(v - n_old) * d, d);
                if (!(dv > bd[i])) return false;
                bool dup = false;
                for (int t = 0; t < nseen; ++t) dup = dup || seen[t] == v;
                if (!dup) {
                    if (nseen == kSeen) return false;
                    seen[nseen++] = v;
                }
            }
        }
        // The sequential search would have made these extra visits.
        return nseen == 0 || (sl_st[slot] == ROAR_OK && (uint64_t)sl_vis[slot] + (uint64_t)nseen < kMaxVisits);
    }

    void mark_changed(int64_t r) {
        stamp[r] = applied;
        if (!chg_mark[r]) {
            chg_mark[r] = 1;
            chg.push_back(r);
        }
    }

    // Steps 2-3 for the given slots: the first pool entry with a connected
    // query, then (nearest_query) the connected query nearest to the row.
    std::vector<int64_t> hcoff;
    std::vector<uint32_t> hcids;
    std::vector<int> pick_slots;
    roar_status pick_queries(const std::vector<int> &slots) {
        pick_slots.clear();
        hxs_pick.clear();
        hcoff.assign(1, 0);
        hcids.clear();
        for (int slot : slots) {
            const uint32_t *pool = sl_pool.data() + (size_t)slot * L;
            sl_q[slot] = -1;
            for (int r = 0; r < L && pool[r] != ROAR_NONE_ID; ++r) {
                const uint32_t b = pool[r];
                const size_t before = hcids.size();
                hcids.insert(hcids.end(), inc_ids.begin() + inc_off[b], inc_ids.begin() + inc_off[b + 1]);
                if (b >= n_old) hcids.insert(hcids.end(), inc_new[b - n_old].begin(), inc_new[b - n_old].end());
                if (hcids.size() > before) {
                    pick_slots.push_back(slot);
                    hxs_pick.push_back((uint32_t)sl_v[slot]);
                    hcoff.push_back((int64_t)hcids.size());
                    break;
                }
            }
        }
        const int64_t m = (int64_t)pick_slots.size();
        if (m == 0) return ROAR_OK;
        cudaError_t e = cudaSuccess;
        if ((int64_t)hcids.size() > cids_cap) {
            cudaFree(dcids);
            dcids = nullptr;
            cids_cap = std::max<int64_t>((int64_t)hcids.size(), 2 * cids_cap);
            e = dalloc(&dcids, (size_t)cids_cap);
            if (e != cudaSuccess) {
                cids_cap = 0;
                return fail(e, "roar_insert: connected-query buffer");
            }
        }
        e = cudaMemcpyAsync(dcids, hcids.data(), hcids.size() * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dcoff, hcoff.data(), (size_t)(m + 1) * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dxs_pick, hxs_pick.data(), (size_t)m * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail(e, "roar_insert: query-pick inputs");
        nearest_query<<<(unsigned)m, 256, 0, s>>>(X_dev, dT, d, dxs_pick, dcoff, dcids, dbest);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(hbest.data(), dbest, (size_t)m * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(e, "roar_insert: query pick");
        for (int64_t i = 0; i < m; ++i) sl_q[pick_slots[i]] = hbest[i] == ROAR_NONE_ID ? -1 : (int64_t)hbest[i];
        return ROAR_OK;
    }

    // Alg. 3 (roar_acquire, fill) for nx nodes: xs[i] with candidate row i of
    // hbuf [nx][stride] (nc[i] entries), bound `bound`; results to hout/hcnt.
    roar_status acquire(int64_t nx, int stride, int bound) {
        cudaError_t e = cudaMemcpyAsync(dcand, hbuf.data(), (size_t)nx * stride * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dxs, hxs.data(), (size_t)nx * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dnc, hnc.data(), (size_t)nx * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail(e, "roar_insert: acquire inputs");
        roar_status rc = roar_acquire(X_dev, n_total, d, dxs, nx, dcand, stride, dnc, bound, 1, dout, dcnt,
                                      nullptr, s);
        if (rc != ROAR_OK) return rc;
        e = cudaMemcpyAsync(hout.data(), dout, (size_t)nx * bound * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hcnt.data(), dcnt, (size_t)nx * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(e, "roar_insert: acquire");
        for (int64_t i = 0; i < nx; ++i)
            if (hcnt[i] < 0) {
                set_error("roar_insert: an id outside the base set");
                return ROAR_EINVAL;
            }
        return ROAR_OK;
    }

    // Step 4 for the given slots, from N_out(q) as it stands (or the pool).
    roar_status acquire_lists(const std::vector<int> &slots) {
        for (size_t lo = 0; lo < slots.size(); lo += (size_t)acq_cap) {
            const int64_t nx = std::min<int64_t>(acq_cap, (int64_t)(slots.size() - lo));
            for (int64_t i = 0; i < nx; ++i) {
                const int slot = slots[lo + i];
                const int64_t q = sl_q[slot];
                uint32_t *row = hbuf.data() + (size_t)i * CS;
                int m = 0;
                if (q >= 0) {
                    for (int j = 0; j < nout_cnt[q]; ++j) row[m++] = nout[q * nout_cap + j];
                } else {
                    const uint32_t *pool = sl_pool.data() + (size_t)slot * L;
                    for (int r = 0; r < L && pool[r] != ROAR_NONE_ID; ++r) row[m++] = pool[r];
                }
                std::fill(row + m, row + CS, ROAR_NONE_ID);
                hxs[i] = (uint32_t)sl_v[slot];
                hnc[i] = m;
            }
            roar_status rc = acquire(nx, CS, M);
            if (rc != ROAR_OK) return rc;
            for (int64_t i = 0; i < nx; ++i) {
                const int slot = slots[lo + i];
                std::copy(hout.data() + (size_t)i * M, hout.data() + (size_t)(i + 1) * M,
                          sl_acq.data() + (size_t)slot * M);
                sl_acq_n[slot] = hcnt[i];
                sl_acq_from[slot] = sl_q[slot] >= 0 ? nout_cnt[sl_q[slot]] : -1;
                sl_acq_ok[slot] = 1;
            }
            stats[2] += (double)nx;
        }
        return ROAR_OK;
    }

    // Step 5's re-prunes of full rows, batched: each pending row p becomes
    // Alg. 3 over its row plus the new row recorded in hbuf.
    std::vector<uint32_t> pend_cand;
    roar_status flush_prunes() {
        if (pend.empty()) return ROAR_OK;
        const auto t0 = Clock::now();
        const int64_t nf = (int64_t)pend.size();
        std::copy(pend_cand.begin(), pend_cand.begin() + (size_t)nf * (R + 1), hbuf.begin());
        for (int64_t i = 0; i < nf; ++i) {
            hxs[i] = (uint32_t)pend[i];
            hnc[i] = R + 1;
        }
        roar_status rc = acquire(nf, R + 1, R);
        if (rc != ROAR_OK) return rc;
        for (int64_t i = 0; i < nf; ++i) {
            uint32_t *rp = adj.data() + (size_t)pend[i] * R;
            for (int t = 0; t < R; ++t) rp[t] = t < hcnt[i] ? hout[(size_t)i * R + t] : ROAR_NONE_ID;
            pend_mark[pend[i]] = 0;
        }
        stats[4] += 1;
        stats[5] += (double)nf;
        stats[10] += since(t0);
        pend.clear();
        return ROAR_OK;
    }

    roar_status scatter() {
        for (size_t lo = 0; lo < chg.size(); lo += (size_t)chg_cap) {
            const int64_t m = std::min<int64_t>(chg_cap, (int64_t)(chg.size() - lo));
            for (int64_t i = 0; i < m; ++i) {
                const int64_t r = chg[lo + i];
                std::copy(adj.data() + (size_t)r * R, adj.data() + (size_t)(r + 1) * R, hbuf.data() + (size_t)i * R);
                hdst[i] = r;
            }
            cudaError_t e = cudaMemcpyAsync(drows, hbuf.data(), (size_t)m * R * 4, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(ddst, hdst.data(), (size_t)m * 8, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return fail(e, "roar_insert: scatter inputs");
            const int64_t total = m * R;
            scatter_rows<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(adj_dev, R, drows, ddst, m);
            e = cudaGetLastError();
            // the host buffers are reused at once: wait for the copies
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return fail(e, "roar_insert: scatter");
        }
        for (int64_t r : chg) chg_mark[r] = 0;
        chg.clear();
        return ROAR_OK;
    }

    // Step 1 for the given slots: one launch on the graph as it stands.
    roar_status search(const std::vector<int> &slots) {
        const int64_t m = (int64_t)slots.size();
        for (int64_t i = 0; i < m; ++i)
            std::memcpy(hq.data() + (size_t)i * d, Xnew.data() + (size_t)(sl_v[slots[i]] - n_old) * d,
                        (size_t)d * 4);
        cudaError_t e = cudaMemcpyAsync(dq, hq.data(), (size_t)m * d * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail(e, "roar_insert: queries");
        // Few queries: teams of warps per query shorten the launch (results
        // never depend on the team width).
        const int tw = m <= 48 ? 8 : m <= 128 ? 4 : m <= 384 ? 2 : 1;
        roar_status rc = roar_index_set_tuning(gi, L, tw, 0, 0);
        if (rc != ROAR_OK) return rc;
        SearchArgs a;
        int blocks = 0, tw_plan = 1;
        rc = plan_search(gi, L, a, blocks, tw_plan, m);
        if (rc != ROAR_OK) return rc;
        a.q = dq;
        a.nq = m;
        a.k = L;
        a.L = L;
        a.ids = dids;
        a.dist = ddist;
        a.hops = dhops;
        a.qstatus = dst;
        a.visits = dvis;
        a.trace = dtrace;
        a.trace_bound = dbound;
        a.trace_cap = TC;
        e = launch_search(a, blocks, tw_plan, s);
        if (e != cudaSuccess) return fail(e, "roar_insert: search launch");
        std::vector<uint32_t> ids((size_t)m * L), hops((size_t)m), tr((size_t)m * TC), vis((size_t)m);
        std::vector<float> bnd((size_t)m * TC);
        std::vector<int32_t> st((size_t)m);
        e = cudaMemcpyAsync(ids.data(), dids, ids.size() * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hops.data(), dhops, hops.size() * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tr.data(), dtrace, tr.size() * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bnd.data(), dbound, bnd.size() * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vis.data(), dvis, vis.size() * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(st.data(), dst, st.size() * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(e, "roar_insert: search");
        for (int64_t i = 0; i < m; ++i) {
            const int slot = slots[i];
            std::copy(ids.begin() + (size_t)i * L, ids.begin() + (size_t)(i + 1) * L,
                      sl_pool.begin() + (size_t)slot * L);
            std::copy(tr.begin() + (size_t)i * TC, tr.begin() + (size_t)(i + 1) * TC,
                      sl_trace.begin() + (size_t)slot * TC);
            std::copy(bnd.begin() + (size_t)i * TC, bnd.begin() + (size_t)(i + 1) * TC,
                      sl_bound.begin() + (size_t)slot * TC);
            sl_hops[slot] = hops[i];
            sl_vis[slot] = vis[i];
            sl_st[slot] = st[i];
            sl_snap[slot] = applied;
            sl_q[slot] = -2;
            sl_acq_ok[slot] = 0;
        }
        stats[1] += (double)m;
        return ROAR_OK;
    }

    // Steps 5-6 for row v (its list N(v) in the slot).
    roar_status apply(int slot, int64_t v) {
        const int nr = sl_acq_n[slot];
        const int64_t q = sl_q[slot];
        uint32_t *rowv = adj.data() + (size_t)v * R;
        const uint32_t *nv = sl_acq.data() + (size_t)slot * M;
        for (int j = 0; j < R; ++j) rowv[j] = j < nr ? nv[j] : ROAR_NONE_ID;
        mark_changed(v);
        rewrite[v] = applied;
        for (int j = 0; j < nr; ++j) {
            const uint32_t p = rowv[j];
            if (pend_mark[p]) {
                roar_status rc = flush_prunes();
                if (rc != ROAR_OK) return rc;
            }
            uint32_t *rp = adj.data() + (size_t)p * R;
            int deg = 0;
            bool has = false;
            while (deg < R && rp[deg] != ROAR_NONE_ID) has |= rp[deg++] == (uint32_t)v;
            if (has) continue;
            mark_changed(p);
            if (deg < R) {
                rp[deg] = (uint32_t)v;
                pos_seq[(size_t)p * R + deg] = (int32_t)applied;
                continue;
            }
            if ((int64_t)pend.size() == acq_cap) {
                roar_status rc = flush_prunes();
                if (rc != ROAR_OK) return rc;
            }
            uint32_t *c = pend_cand.data() + pend.size() * (size_t)(R + 1);
            std::copy(rp, rp + R, c);
            c[R] = (uint32_t)v;
            rewrite[p] = applied;
            pend.push_back(p);
            pend_mark[p] = 1;
        }
        if (q >= 0 && nout_cnt[q] < nout_cap) {
            nout[q * nout_cap + nout_cnt[q]++] = (uint32_t)v;
            inc_new[v - n_old].push_back((uint32_t)q);
        }
        chosen_q[v - n_old] = (int32_t)q;
        ++applied;
        sl_snap[slot] = -1;
        sl_v[slot] = -1;
        return ROAR_OK;
    }

    roar_status run(const uint32_t *pivot) {
        const auto t_setup = Clock::now();
        const int64_t n_new = n_total - n_old;
        adj.resize((size_t)n_total * R);
        Xnew.resize((size_t)n_new * d);
        cudaError_t e = cudaMemcpyAsync(adj.data(), adj_dev, adj.size() * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(Xnew.data(), X_dev + (size_t)n_old * d, Xnew.size() * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(e, "roar_insert: copy graph");
        inc_off.assign((size_t)n_total + 1, 0);
        for (int64_t t = 0; t < nt; ++t) {
            if (pivot[t] < n_total) ++inc_off[pivot[t] + 1];
            for (int j = 0; j < nout_cnt[t]; ++j) {
                const uint32_t b = nout[t * nout_cap + j];
                if (b < n_total) ++inc_off[b + 1];
            }
        }
        for (int64_t b = 0; b < n_total; ++b) inc_off[b + 1] += inc_off[b];
        inc_ids.resize((size_t)inc_off[n_total]);
        {
            std::vector<int64_t> fill(inc_off.begin(), inc_off.end() - 1);
            for (int64_t t = 0; t < nt; ++t) {
                if (pivot[t] < n_total) inc_ids[fill[pivot[t]]++] = (uint32_t)t;
                for (int j = 0; j < nout_cnt[t]; ++j) {
                    const uint32_t b = nout[t * nout_cap + j];
                    if (b < n_total) inc_ids[fill[b]++] = (uint32_t)t;
                }
            }
        }
        inc_new.assign((size_t)n_new, {});
        stamp.assign((size_t)n_total, -1);
        rewrite.assign((size_t)n_total, -1);
        pos_seq.assign((size_t)n_total * R, -1);
        pend_mark.assign((size_t)n_total, 0);
        chg_mark.assign((size_t)n_total, 0);
        TC = 2 * L + 128;
        CS = std::max(std::max(nout_cap, L), R + 1);
        acq_cap = std::max<int64_t>(W, 256);
        chg_cap = (int64_t)W * (M + 1) + 1;
        sl_v.assign(W, -1);
        sl_snap.assign(W, -1);
        sl_q.assign(W, -2);
        sl_hops.assign(W, 0);
        sl_pool.assign((size_t)W * L, ROAR_NONE_ID);
        sl_trace.assign((size_t)W * TC, 0);
        sl_bound.assign((size_t)W * TC, 0.0f);
        sl_vis.assign(W, 0);
        sl_st.assign(W, 0);
        sl_acq.assign((size_t)W * M, ROAR_NONE_ID);
        sl_acq_n.assign(W, 0);
        sl_acq_from.assign(W, -1);
        sl_acq_ok.assign(W, 0);
        pend_cand.assign((size_t)acq_cap * (R + 1), ROAR_NONE_ID);
        hq.resize((size_t)W * d);
        hbuf.resize(std::max((size_t)acq_cap * CS, (size_t)chg_cap * R));
        hxs.resize((size_t)acq_cap);
        hnc.resize((size_t)acq_cap);
        hcnt.resize((size_t)acq_cap);
        hout.resize((size_t)acq_cap * R);
        hdst.resize((size_t)chg_cap);
        e = dalloc(&dq, (size_t)W * d);
        if (e == cudaSuccess) e = dalloc(&ddist, (size_t)W * L);
        if (e == cudaSuccess) e = dalloc(&dids, (size_t)W * L);
        if (e == cudaSuccess) e = dalloc(&dhops, (size_t)W);
        if (e == cudaSuccess) e = dalloc(&dst, (size_t)W);
        if (e == cudaSuccess) e = dalloc(&dtrace, (size_t)W * TC);
        if (e == cudaSuccess) e = dalloc(&dbound, (size_t)W * TC);
        if (e == cudaSuccess) e = dalloc(&dvis, (size_t)W);
        if (e == cudaSuccess) e = dalloc(&dxs, (size_t)acq_cap);
        if (e == cudaSuccess) e = dalloc(&dcand, (size_t)acq_cap * CS);
        if (e == cudaSuccess) e = dalloc(&dnc, (size_t)acq_cap);
        if (e == cudaSuccess) e = dalloc(&dout, (size_t)acq_cap * R);
        if (e == cudaSuccess) e = dalloc(&dcnt, (size_t)acq_cap);
        if (e == cudaSuccess) e = dalloc(&drows, (size_t)chg_cap * R);
        if (e == cudaSuccess) e = dalloc(&ddst, (size_t)chg_cap);
        if (e == cudaSuccess) e = dalloc(&dT, (size_t)nt * d);
        if (e == cudaSuccess) e = dalloc(&dxs_pick, (size_t)W);
        if (e == cudaSuccess) e = dalloc(&dbest, (size_t)W);
        if (e == cudaSuccess) e = dalloc(&dcoff, (size_t)W + 1);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("roar_insert: out of device memory");
            return ROAR_ENOMEM;
        }
        hbest.resize((size_t)W);
        e = cudaMemcpyAsync(dT, T, (size_t)nt * d * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail(e, "roar_insert: training queries");
        roar_status rc = roar_index_create(n_total, d, X_dev, ROAR_F32, nullptr, nullptr, adj_dev, R, entry,
                                           kMaxVisits, &gi);
        if (rc != ROAR_OK) return rc;
        stats[6] = since(t_setup);
        std::vector<int> need, acq;
        for (int64_t head = n_old; head < n_total;) {
            const int64_t end = std::min<int64_t>(head + W, n_total);
            stats[0] += 1;
            // 1. searches for the window rows without a usable result
            need.clear();
            for (int64_t v = head; v < end; ++v) {
                const int slot = (int)(v % W);
                if (sl_v[slot] != v) {
                    sl_v[slot] = v;
                    sl_snap[slot] = -1;
                }
                if (!usable(slot)) need.push_back(slot);
            }
            if (!need.empty()) {
                const auto t0 = Clock::now();
                rc = search(need);
                if (rc != ROAR_OK) return rc;
                stats[7] += since(t0);
            }
            // 2-4. connected query and N(v), where missing or stale
            acq.clear();
            for (int64_t v = head; v < end; ++v)
                if (sl_q[(int)(v % W)] == -2) acq.push_back((int)(v % W));
            if (!acq.empty()) {
                const auto t0 = Clock::now();
                rc = pick_queries(acq);
                if (rc != ROAR_OK) return rc;
                stats[12] += since(t0);
            }
            acq.clear();
            for (int64_t v = head; v < end; ++v) {
                const int slot = (int)(v % W);
                const int32_t from = sl_q[slot] >= 0 ? nout_cnt[sl_q[slot]] : -1;
                if (!sl_acq_ok[slot] || sl_acq_from[slot] != from) acq.push_back(slot);
            }
            if (!acq.empty()) {
                const auto t0 = Clock::now();
                rc = acquire_lists(acq);
                if (rc != ROAR_OK) return rc;
                stats[8] += since(t0);
            }
            const auto t_apply = Clock::now();
            // 5-6. apply in order while the searches are exact
            int64_t v = head;
            for (; v < end; ++v) {
                const int slot = (int)(v % W);
                if (!usable(slot)) {
                    bool rewritten = sl_hops[slot] > (uint32_t)TC;
                    const uint32_t *tr = sl_trace.data() + (size_t)slot * TC;
                    for (uint32_t i = 0; !rewritten && i < sl_hops[slot]; ++i)
                        rewritten = rewrite[tr[i]] >= sl_snap[slot];
                    stats[rewritten ? 13 : 14] += 1;
                    break;
                }
                const int64_t q = sl_q[slot];
                if (q >= 0 && sl_acq_from[slot] != nout_cnt[q]) {   // N_out(q) grew in this window
                    rc = acquire_lists(std::vector<int>{slot});
                    if (rc != ROAR_OK) return rc;
                    stats[3] += 1;
                }
                rc = apply(slot, v);
                if (rc != ROAR_OK) return rc;
            }
            rc = flush_prunes();
            if (rc != ROAR_OK) return rc;
            stats[9] += since(t_apply);
            const auto t_sc = Clock::now();
            rc = scatter();
            if (rc != ROAR_OK) return rc;
            stats[11] += since(t_sc);
            head = v;
        }
        return ROAR_OK;
    }

    ~Inserter() {
        if (gi) roar_index_destroy(gi);
        cudaFree(dq);
        cudaFree(ddist);
        cudaFree(dids);
        cudaFree(dhops);
        cudaFree(dst);
        cudaFree(dtrace);
        cudaFree(dbound);
        cudaFree(dvis);
        cudaFree(dxs);
        cudaFree(dcand);
        cudaFree(dnc);
        cudaFree(dout);
        cudaFree(dcnt);
        cudaFree(drows);
        cudaFree(ddst);
        cudaFree(dT);
        cudaFree(dcids);
        cudaFree(dxs_pick);
        cudaFree(dbest);
        cudaFree(dcoff);
    }
};

}  // namespace

extern "C" roar_status roar_insert(const float *X_dev, int64_t n_total, int32_t d, uint32_t *adj_dev, int32_t R,
                                   uint32_t entry, int64_t n_old, const float *T_host, int64_t nt,
                                   const uint32_t *pivot_host, uint32_t *nout_host, int32_t *nout_cnt_host,
                                   int32_t nout_cap, int32_t M, int32_t L, int32_t window, int32_t *chosen_q_host,
                                   double *stats, void *stream) {
    if (!X_dev || !adj_dev || !T_host || !pivot_host || !nout_host || !nout_cnt_host || !chosen_q_host ||
        n_old < 1 || n_total < n_old || n_total >= 0x7FFFFFFF || (int64_t)entry >= n_old || d < 4 || d % 4 ||
        d > 1024 || R < 1 || R > 64 || M < 1 || M > R || L < 1 || L > ROAR_MAX_L || nt < 1 || nout_cap < 1 ||
        nout_cap > 1024 || window < 1 || window > 4096) {
        set_error("roar_insert: bad arguments (need n_old >= 1, entry < n_old, d % 4 == 0, 1 <= M <= R <= 64, "
                  "L <= ROAR_MAX_L, nout_cap <= 1024, 1 <= window <= 4096)");
        return ROAR_EINVAL;
    }
    if (stats)
        for (int i = 0; i < Inserter::kStats; ++i) stats[i] = 0.0;
    if (n_total == n_old) return ROAR_OK;
    Inserter ins;
    ins.X_dev = X_dev;
    ins.n_total = n_total;
    ins.n_old = n_old;
    ins.d = d;
    ins.R = R;
    ins.M = M;
    ins.L = L;
    ins.W = window;
    ins.T = T_host;
    ins.nt = nt;
    ins.entry = entry;
    ins.nout_cap = nout_cap;
    ins.nout = nout_host;
    ins.nout_cnt = nout_cnt_host;
    ins.chosen_q = chosen_q_host;
    ins.adj_dev = adj_dev;
    ins.s = (cudaStream_t)stream;
    roar_status rc = ins.run(pivot_host);
    cudaError_t e = cudaStreamSynchronize(ins.s);
    if (stats)
        for (int i = 0; i < Inserter::kStats; ++i) stats[i] = ins.stats[i];
    if (rc == ROAR_OK && e != cudaSuccess) return cuda_fail(e, "roar_insert");
    return rc;
}
