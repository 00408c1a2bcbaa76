// Serving loop: continuous batching of search requests into one persistent
// search kernel (no counterpart in the paper, which measures single-thread
// search latency; the per-query search is the paper's beam search, Sec. 4.3).
//
// Requests live in a ring of query slots in device memory. Every exchange
// with the host goes through the copy engines, never through host memory the
// kernel reads or writes (under load, the GPU saw the host's writes to mapped
// host memory, and the host saw the GPU's, up to a second late):
//   - submit writes each query's record (query, k, L) and publish mark (the
//     low 32 bits of its sequence number + 1) into pinned staging slots; the
//     poller thread copies every newly staged range to the device ring, the
//     records first and then, by a later copy in the same stream, the marks
//     (a few copies per poll round, however many requests arrived; a copy
//     per array and request kept the copy engine and the teams waiting);
//   - the kernel's teams take tickets (sequence numbers) in order with an
//     atomicAdd on a device head counter, wait for the ticket's slot to be
//     published, search, write the results into the slot and then the slot's
//     done mark; when no ticket has been served for idle_ms the whole kernel
//     exits, each team keeping its ticket for the next launch;
//   - a host poller thread copies the done marks of the slots in flight to a
//     pinned shadow, timestamps completions and relaunches the kernel when
//     work is pending but the kernel has exited (its teams exit after a
//     bounded idle period, so no launch can wait forever);
//   - poll copies a complete request's results to the caller and releases
//     its slots.
// Admission: a request is taken only if the ring has room for all its queries
// and, under a memory budget, if its charge fits beside the requests in
// flight. A query at (k, L) is charged its ring bytes at its own k (query 4d,
// results 8k, counters 24), its candidate pool (8L) and the exact visited
// table a beam of width L needs (2^ceil(log2(32 L)) slots of 4 bytes, the
// kernel's own sizing rule for its shared-memory table); a request gives its
// charge back when it is released.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "roar_internal.cuh"

namespace roar {
roar_status cuda_fail(cudaError_t e, const char *what);
void set_error(const char *msg);
}  // namespace roar

using namespace roar;

namespace {
using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t first;   // sequence number of its first query
    int32_t nq, k;
    int64_t charge = 0;   // bytes charged against the memory budget
    Clock::time_point t_submit, t_done;
    int32_t checked = 0;  // queries already seen done
    bool complete = false, polling = false, released = false;
};

template <class T>
cudaError_t dev_alloc(T **d, size_t count) {
    cudaError_t e = cudaMalloc((void **)d, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) e = cudaMemset(*d, 0, std::max<size_t>(count, 1) * sizeof(T));
    return e;
}

template <class T>
cudaError_t host_pinned(T **h, size_t count) {
    cudaError_t e = cudaMallocHost((void **)h, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) std::memset((void *)*h, 0, std::max<size_t>(count, 1) * sizeof(T));
    return e;
}
}  // namespace

struct roar_server {
    roar_index *idx = nullptr;
    int32_t d = 0, k_max = 0, L_max = 0, tw = 1;
    int64_t R = 0;
    uint32_t idle_polls = 50000;
    // device ring: per slot a record of `stride` floats (query, k, L, padding)
    int32_t stride = 0;
    float *rec_d = nullptr;
    uint32_t *pub_d = nullptr, *done_d = nullptr;
    uint32_t *ids_d = nullptr, *vis_d = nullptr, *hops_d = nullptr;
    float *dist_d = nullptr;
    int32_t *st_d = nullptr;
    int *stop_d = nullptr;
    unsigned long long *head_dev = nullptr;
    unsigned long long *orphan_d = nullptr;   // per team slot (see the kernel's claim)
    unsigned long long *clock_d = nullptr;    // the kernel's idle clock and closing flag
    // pinned host staging (submit) and the poller's shadow of the done marks
    float *rec_h = nullptr;
    uint32_t *pub_h = nullptr, *done_h = nullptr;
    int *one_h = nullptr;   // the stop value, 1
    // pinned copies of the result rings (poll reads a request's slots here)
    uint32_t *rids_h = nullptr, *rvis_h = nullptr;
    float *rdist_h = nullptr;
    int32_t *rst_h = nullptr;
    cudaStream_t stream = nullptr;       // the persistent kernel
    cudaStream_t in_stream = nullptr;    // staged records, then their marks (stream order)
    cudaStream_t mark_stream = nullptr;  // the poller's done-mark copies
    cudaStream_t res_stream = nullptr;   // poll's result copies
    cudaEvent_t ev_end = nullptr;
    SearchArgs args;
    int blocks = 0;
    bool launched = false;
    bool running = false;     // the kernel was running when last asked
    int64_t launches = 0;
    // host bookkeeping
    std::mutex mu;
    std::mutex res_mu;        // serialises poll's use of res_stream
    uint64_t tail = 0;        // queries staged by submit
    uint64_t published = 0;   // queries whose records and marks the poller has copied
    uint64_t released = 0;    // queries whose slots are free again
    uint64_t completed_q = 0;
    int64_t budget = 0;       // bytes of in-flight requests allowed (0: slots only)
    int64_t inflight = 0;     // bytes charged to requests not yet released
    std::deque<Request> reqs; // submission order, trimmed when released
    std::atomic<bool> quit{false};
    std::thread poller;
};

namespace {

// Bytes one query at (k, L) is charged: ring slot at its own k, candidate pool
// and the exact visited table for a beam of width L.
int64_t query_charge(int32_t d, int32_t k, int32_t L) {
    int lg = 0;
    while ((1ll << lg) < 32ll * L) ++lg;
    return 4ll * d + 8ll * k + 24 + 8ll * L + (4ll << lg);
}

bool kernel_running(roar_server *s) {
    if (!s->launched) return false;
    return cudaEventQuery(s->ev_end) == cudaErrorNotReady;
}

roar_status launch_locked(roar_server *s) {
    // A new launch starts with the idle clock cleared and not closing.
    cudaError_t e = cudaMemsetAsync(s->clock_d, 0, 2 * sizeof(unsigned long long), s->stream);
    if (e == cudaSuccess) e = launch_search(s->args, s->blocks, s->tw, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_end, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "roar_server: launch");
    s->launched = true;
    s->running = true;
    ++s->launches;
    return ROAR_OK;
}

// Copy ring elements [a, b) (sequence numbers, taken mod R; `width` values
// each) between a device ring and a pinned host ring, in at most two copies.
template <class T>
cudaError_t copy_ring(T *dst, const T *src, uint64_t a, uint64_t b, int64_t R, size_t width, cudaMemcpyKind kind,
                      cudaStream_t st) {
    if (b <= a) return cudaSuccess;
    const uint64_t s0 = a % (uint64_t)R;
    const uint64_t n = b - a;
    const uint64_t n1 = std::min<uint64_t>(n, (uint64_t)R - s0);
    cudaError_t e = cudaMemcpyAsync(dst + s0 * width, src + s0 * width, n1 * width * sizeof(T), kind, st);
    if (e == cudaSuccess && n > n1) e = cudaMemcpyAsync(dst, src, (n - n1) * width * sizeof(T), kind, st);
    return e;
}

// The poller works on a snapshot of the incomplete requests: the lock is held
// only to copy it and to apply what the done marks showed, so submit, poll and
// ready do not wait behind the copy of the marks. Incomplete requests are
// never released, so each snapshot entry is still in the list when its update
// is applied. The kernel's state is asked of the driver (an event query) only
// while work is waiting, and at most every 100 us.
void poll_loop(roar_server *s) {
    struct Pending {
        uint64_t first;
        int32_t nq, checked, now_checked;
    };
    std::vector<Pending> snap;
    Clock::time_point last_query = Clock::now();
    while (!s->quit.load(std::memory_order_acquire)) {
        snap.clear();
        uint64_t hi = 0, pub_lo = 0;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            for (const Request &r : s->reqs)
                if (!r.complete) snap.push_back({r.first, r.nq, r.checked, r.checked});
            hi = s->tail;
            pub_lo = s->published;
        }
        if (hi > pub_lo) {
            // Publish what submit staged since the last round: records, then
            // marks. The staging of these slots is not rewritten before the
            // slots are released, which needs their queries done.
            cudaError_t e = copy_ring(s->rec_d, s->rec_h, pub_lo, hi, s->R, (size_t)s->stride,
                                      cudaMemcpyHostToDevice, s->in_stream);
            if (e == cudaSuccess)
                e = copy_ring(s->pub_d, s->pub_h, pub_lo, hi, s->R, 1, cudaMemcpyHostToDevice, s->in_stream);
            if (e == cudaSuccess) {
                std::lock_guard<std::mutex> lock(s->mu);
                s->published = hi;
            }
        }
        bool any = false;
        if (!snap.empty()) {
            // Done marks of every sequence number from the oldest unchecked one
            // to the tail (at most R slots), into the pinned shadow.
            const uint64_t lo = snap.front().first + (uint64_t)snap.front().checked;
            cudaError_t e = copy_ring(s->done_h, s->done_d, lo, hi, s->R, 1, cudaMemcpyDeviceToHost, s->mark_stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->mark_stream);
            if (e == cudaSuccess) {
                for (Pending &p : snap) {
                    while (p.now_checked < p.nq) {
                        const uint64_t seq = p.first + (uint64_t)p.now_checked;
                        if (s->done_h[seq % (uint64_t)s->R] != (uint32_t)(seq + 1)) break;
                        ++p.now_checked;
                    }
                    any = any || p.now_checked != p.checked;
                }
            }
        }
        const Clock::time_point now = Clock::now();
        {
            std::lock_guard<std::mutex> lock(s->mu);
            if (any) {
                for (const Pending &p : snap) {
                    if (p.now_checked == p.checked) continue;
                    auto it = std::lower_bound(s->reqs.begin(), s->reqs.end(), p.first,
                                               [](const Request &x, uint64_t id) { return x.first < id; });
                    if (it == s->reqs.end() || it->first != p.first) continue;
                    s->completed_q += (uint64_t)(p.now_checked - it->checked);
                    it->checked = p.now_checked;
                    if (it->checked == it->nq) {
                        it->complete = true;
                        it->t_done = now;
                    }
                }
            }
            // Teams exit after an idle period: relaunch if work is waiting.
            if (s->completed_q < s->published && now - last_query > std::chrono::microseconds(100)) {
                last_query = now;
                s->running = kernel_running(s);
                if (!s->running) launch_locked(s);
            }
        }
        std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
}

}  // namespace

extern "C" roar_status roar_server_create(roar_index *idx, const roar_server_cfg *cfg, roar_server **out) {
    if (!out || !idx || !cfg || cfg->k_max < 1 || cfg->L_max < cfg->k_max || cfg->L_max > ROAR_MAX_L ||
        cfg->ring_capacity < 0 || cfg->memory_budget < 0 || cfg->idle_ms < 0 ||
        (cfg->team_warps != 0 && cfg->team_warps != 1 && cfg->team_warps != 2 && cfg->team_warps != 4 &&
         cfg->team_warps != 8)) {
        set_error("roar_server_create: bad configuration");
        return ROAR_EINVAL;
    }
    *out = nullptr;
    roar_server *s = new (std::nothrow) roar_server();
    if (!s) return ROAR_ENOMEM;
    s->idx = idx;
    s->k_max = cfg->k_max;
    s->L_max = cfg->L_max;
    SearchArgs &a = s->args;
    roar_status st = ROAR_OK;
    if (cfg->team_warps) st = roar_index_set_tuning(idx, cfg->L_max, cfg->team_warps, 0, 0);
    if (st == ROAR_OK) st = plan_search(idx, cfg->L_max, a, s->blocks, s->tw, (int64_t)1 << 40);
    if (st != ROAR_OK) {
        delete s;
        return st;
    }
    s->d = a.d;
    // Ring capacity: given, or as many k_max-wide slots as the budget could
    // hold; the budget itself is enforced per request at submission.
    const int64_t slot_bytes = (int64_t)s->d * 4 + (int64_t)s->k_max * 8 + 24;
    s->budget = cfg->memory_budget;
    s->R = cfg->ring_capacity ? cfg->ring_capacity
                              : (cfg->memory_budget ? std::min<int64_t>((int64_t)1 << 26, cfg->memory_budget / slot_bytes)
                                                    : 65536);
    if (s->R < 1 || s->R > ((int64_t)1 << 26)) {
        set_error("roar_server_create: ring capacity must be 1..2^26 queries");
        delete s;
        return ROAR_EINVAL;
    }
    s->idle_polls = (uint32_t)((cfg->idle_ms ? cfg->idle_ms : 50) * 1000);
    const size_t R = (size_t)s->R;
    s->stride = s->d + 4;   // d % 4 == 0: records stay 16-byte aligned
    cudaError_t e = dev_alloc(&s->rec_d, R * s->stride);
    if (e == cudaSuccess) e = dev_alloc(&s->pub_d, R);
    if (e == cudaSuccess) e = dev_alloc(&s->done_d, R);
    if (e == cudaSuccess) e = dev_alloc(&s->ids_d, R * s->k_max);
    if (e == cudaSuccess) e = dev_alloc(&s->dist_d, R * s->k_max);
    if (e == cudaSuccess) e = dev_alloc(&s->vis_d, R);
    if (e == cudaSuccess) e = dev_alloc(&s->hops_d, R);
    if (e == cudaSuccess) e = dev_alloc(&s->st_d, R);
    if (e == cudaSuccess) e = dev_alloc(&s->stop_d, 1);
    if (e == cudaSuccess) e = dev_alloc(&s->head_dev, 1);
    const size_t team_slots = (size_t)s->blocks * (size_t)teams_per_block(s->tw);
    if (e == cudaSuccess) e = dev_alloc(&s->orphan_d, team_slots);
    if (e == cudaSuccess) e = cudaMemset(s->orphan_d, 0xFF, team_slots * sizeof(unsigned long long));
    if (e == cudaSuccess) e = dev_alloc(&s->clock_d, 2);
    if (e == cudaSuccess) e = host_pinned(&s->rec_h, R * s->stride);
    if (e == cudaSuccess) e = host_pinned(&s->pub_h, R);
    if (e == cudaSuccess) e = host_pinned(&s->done_h, R);
    if (e == cudaSuccess) e = host_pinned(&s->one_h, 1);
    if (e == cudaSuccess) e = host_pinned(&s->rids_h, R * s->k_max);
    if (e == cudaSuccess) e = host_pinned(&s->rdist_h, R * s->k_max);
    if (e == cudaSuccess) e = host_pinned(&s->rvis_h, R);
    if (e == cudaSuccess) e = host_pinned(&s->rst_h, R);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->in_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->mark_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->res_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_end, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        roar_status rc = cuda_fail(e, "roar_server_create");
        roar_server_destroy(s);
        return rc;
    }
    *s->one_h = 1;
    a.nq = (int64_t)1 << 62;
    a.ring_rec = s->rec_d;
    a.ring_stride = s->stride;
    a.ids = s->ids_d;
    a.dist = s->dist_d;
    a.visits = s->vis_d;
    a.hops = s->hops_d;
    a.qstatus = s->st_d;
    a.ring_pub = s->pub_d;
    a.ring_head = s->head_dev;
    a.ring_orphan = s->orphan_d;
    a.ring_clock = s->clock_d;
    a.ring_done = s->done_d;
    a.ring_stop = s->stop_d;
    a.ring_cap = s->R;
    a.ring_kmax = s->k_max;
    a.idle_polls = s->idle_polls;
    s->poller = std::thread(poll_loop, s);
    *out = s;
    return ROAR_OK;
}

extern "C" roar_status roar_server_submit(roar_server *s, const float *q_host, int32_t nq, int32_t k,
                                          int32_t L, uint64_t *request_id) {
    if (!s || !q_host || !request_id || nq < 1 || k < 1 || k > s->k_max || L < k || L > s->L_max) {
        set_error("roar_server_submit: need 1 <= k <= k_max, k <= L <= L_max, nq >= 1");
        return ROAR_EINVAL;
    }
    const int64_t charge = (int64_t)nq * query_charge(s->d, k, L);
    if (s->budget > 0 && charge > s->budget) {
        set_error("roar_server_submit: the request's charge exceeds the whole memory budget");
        return ROAR_EINVAL;
    }
    if (nq > s->R) {
        set_error("roar_server_submit: more queries than ring slots");
        return ROAR_EINVAL;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    // Admission: free ring slots for every query, and room in the budget.
    if ((int64_t)(s->tail - s->released) + nq > s->R) return ROAR_EBUSY;
    if (s->budget > 0 && s->inflight + charge > s->budget) return ROAR_EBUSY;
    const uint64_t first = s->tail, last = first + (uint64_t)nq;
    // Free slots were released after their queries completed, so their
    // staging is no longer being copied. The poller publishes them.
    for (int32_t i = 0; i < nq; ++i) {
        const size_t slot = (size_t)((first + (uint64_t)i) % (uint64_t)s->R);
        float *rec = s->rec_h + slot * (size_t)s->stride;
        std::memcpy(rec, q_host + (size_t)i * s->d, (size_t)s->d * 4);
        int32_t kl[2] = {k, L};
        std::memcpy(rec + s->d, kl, sizeof kl);
        s->pub_h[slot] = (uint32_t)(first + (uint64_t)i + 1);
    }
    s->tail = last;
    Request r;
    r.first = first;
    r.nq = nq;
    r.k = k;
    r.charge = charge;
    s->inflight += charge;
    r.t_submit = Clock::now();
    s->reqs.push_back(r);
    *request_id = first;
    // The kernel is launched, or relaunched after an idle exit, by the poller
    // once the queries are published.
    return ROAR_OK;
}

extern "C" roar_status roar_server_poll(roar_server *s, uint64_t request_id, int32_t timeout_ms,
                                        uint32_t *ids, float *dist, uint32_t *visits, int32_t *qstatus,
                                        double *latency_s) {
    if (!s || timeout_ms < 0) return ROAR_EINVAL;
    const Clock::time_point deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
    uint64_t first = 0;
    int32_t nq = 0, k = 0;
    double lat = 0.0;
    for (;;) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            // reqs is in submission order, so sorted by first query.
            auto it = std::lower_bound(s->reqs.begin(), s->reqs.end(), request_id,
                                       [](const Request &x, uint64_t id) { return x.first < id; });
            if (it == s->reqs.end() || it->first != request_id || it->released || it->polling) {
                set_error("roar_server_poll: unknown or already released request");
                return ROAR_EINVAL;
            }
            if (it->complete) {
                it->polling = true;
                first = it->first;
                nq = it->nq;
                k = it->k;
                lat = std::chrono::duration<double>(it->t_done - it->t_submit).count();
                break;
            }
        }
        if (Clock::now() >= deadline) return ROAR_ETIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
    // The slots stay the request's until it is released below.
    cudaError_t e = cudaSuccess;
    if (ids || dist || visits || qstatus) {
        std::lock_guard<std::mutex> rl(s->res_mu);
        const uint64_t last = first + (uint64_t)nq;
        const size_t km = (size_t)s->k_max;
        if (ids) e = copy_ring(s->rids_h, s->ids_d, first, last, s->R, km, cudaMemcpyDeviceToHost, s->res_stream);
        if (e == cudaSuccess && dist)
            e = copy_ring(s->rdist_h, s->dist_d, first, last, s->R, km, cudaMemcpyDeviceToHost, s->res_stream);
        if (e == cudaSuccess && visits)
            e = copy_ring(s->rvis_h, s->vis_d, first, last, s->R, 1, cudaMemcpyDeviceToHost, s->res_stream);
        if (e == cudaSuccess && qstatus)
            e = copy_ring(s->rst_h, s->st_d, first, last, s->R, 1, cudaMemcpyDeviceToHost, s->res_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->res_stream);
        if (e == cudaSuccess)
            for (int32_t i = 0; i < nq; ++i) {
                const size_t slot = (size_t)((first + (uint64_t)i) % (uint64_t)s->R);
                if (ids) std::memcpy(ids + (size_t)i * k, s->rids_h + slot * km, (size_t)k * 4);
                if (dist) std::memcpy(dist + (size_t)i * k, s->rdist_h + slot * km, (size_t)k * 4);
                if (visits) visits[i] = s->rvis_h[slot];
                if (qstatus) qstatus[i] = s->rst_h[slot];
            }
    }
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = std::lower_bound(s->reqs.begin(), s->reqs.end(), request_id,
                               [](const Request &x, uint64_t id) { return x.first < id; });
    if (e != cudaSuccess) {
        it->polling = false;   // results not delivered: the request stays pollable
        return cuda_fail(e, "roar_server_poll");
    }
    if (latency_s) *latency_s = lat;
    it->released = true;
    s->inflight -= it->charge;
    // Slots free up in ring order.
    while (!s->reqs.empty() && s->reqs.front().released) {
        s->released = s->reqs.front().first + (uint64_t)s->reqs.front().nq;
        s->reqs.pop_front();
    }
    return ROAR_OK;
}

extern "C" roar_status roar_server_ready(roar_server *s, uint64_t *ids, int32_t cap, int32_t *n) {
    if (!s || !n || cap < 0 || (cap > 0 && !ids)) return ROAR_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    int32_t m = 0;
    for (const Request &r : s->reqs) {
        if (m == cap) break;
        if (r.complete && !r.released && !r.polling) ids[m++] = r.first;
    }
    *n = m;
    return ROAR_OK;
}

extern "C" roar_status roar_server_stats(roar_server *s, double *out) {
    if (!s || !out) return ROAR_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    out[0] = (double)s->R;
    out[1] = (double)s->tail;
    out[2] = (double)s->completed_q;
    out[3] = (double)s->released;
    out[4] = (double)s->launches;
    out[5] = (double)s->blocks;
    out[6] = (double)s->tw;
    out[7] = kernel_running(s) ? 1.0 : 0.0;
    out[8] = (double)s->inflight;
    out[9] = (double)s->budget;
    return ROAR_OK;
}

extern "C" void roar_server_destroy(roar_server *s) {
    if (!s) return;
    if (s->stop_d && s->one_h && s->in_stream) {   // ask the teams to exit
        cudaMemcpyAsync(s->stop_d, s->one_h, sizeof(int), cudaMemcpyHostToDevice, s->in_stream);
        cudaStreamSynchronize(s->in_stream);
    }
    if (s->poller.joinable()) {
        s->quit.store(true, std::memory_order_release);
        s->poller.join();
    }
    if (s->stream) cudaStreamSynchronize(s->stream);  // teams exit at their next look at the stop flag
    if (s->ev_end) cudaEventDestroy(s->ev_end);
    for (cudaStream_t st : {s->stream, s->in_stream, s->mark_stream, s->res_stream})
        if (st) cudaStreamDestroy(st);
    cudaFree(s->rec_d);
    cudaFree(s->pub_d);
    cudaFree(s->done_d);
    cudaFree(s->ids_d);
    cudaFree(s->dist_d);
    cudaFree(s->vis_d);
    cudaFree(s->hops_d);
    cudaFree(s->st_d);
    cudaFree(s->stop_d);
    cudaFree(s->head_dev);
    cudaFree(s->orphan_d);
    cudaFree(s->clock_d);
    cudaFreeHost(s->rec_h);
    cudaFreeHost(s->pub_h);
    cudaFreeHost(s->done_h);
    cudaFreeHost(s->one_h);
    cudaFreeHost(s->rids_h);
    cudaFreeHost(s->rdist_h);
    cudaFreeHost(s->rvis_h);
    cudaFreeHost(s->rst_h);
    delete s;
}
