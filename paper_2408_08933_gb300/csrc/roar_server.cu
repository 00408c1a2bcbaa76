// Serving loop: continuous batching of search requests into one persistent
// search kernel (no counterpart in the paper, which measures single-thread
// search latency; the per-query search is the paper's beam search, Sec. 4.3).
//
// Requests live in a ring of query slots in mapped, pinned host memory: the
// host writes a request's queries, k and L into free slots and then publishes
// a new tail; the persistent kernel's teams claim slots one at a time with a
// CAS on a device head counter, read the query coherently, search, write the
// results into the slot and set the slot's done mark after a system fence.
// A host poller thread timestamps completions and relaunches the kernel when
// work is pending but the kernel has exited (its teams exit after a bounded
// idle period, so no launch can wait forever). Admission: a request is taken
// only if the ring has room for all its queries and, under a memory budget,
// if its charge fits beside the requests in flight. A query at (k, L) is
// charged its ring bytes at its own k (query 4d, results 8k, counters 24),
// its candidate pool (8L) and the exact visited table a beam of width L needs
// (2^ceil(log2(32 L)) slots of 4 bytes, the kernel's own sizing rule for its
// shared-memory table); a request gives its charge back when it is released.
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
    bool complete = false, released = false;
};

template <class T>
cudaError_t host_mapped(T **h, T **d, size_t count) {
    cudaError_t e = cudaHostAlloc((void **)h, count * sizeof(T), cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) return e;
    std::memset((void *)*h, 0, count * sizeof(T));
    return cudaHostGetDevicePointer((void **)d, (void *)*h, 0);
}
}  // namespace

struct roar_server {
    roar_index *idx = nullptr;
    int32_t d = 0, k_max = 0, L_max = 0, tw = 1;
    int64_t R = 0;
    uint32_t idle_polls = 50000;
    // ring (host pointer, device pointer)
    float *q_h = nullptr, *q_d = nullptr;
    int32_t *k_h = nullptr, *k_d = nullptr, *L_h = nullptr, *L_d = nullptr;
    uint32_t *ids_h = nullptr, *ids_d = nullptr;
    float *dist_h = nullptr, *dist_d = nullptr;
    uint32_t *vis_h = nullptr, *vis_d = nullptr, *hops_h = nullptr, *hops_d = nullptr;
    int32_t *st_h = nullptr, *st_d = nullptr;
    uint32_t *done_h = nullptr, *done_d = nullptr;
    unsigned long long *tail_h = nullptr, *tail_d = nullptr;
    int *stop_h = nullptr, *stop_d = nullptr;
    unsigned long long *head_dev = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_end = nullptr;
    SearchArgs args;
    int blocks = 0;
    bool launched = false;
    int64_t launches = 0;
    // host bookkeeping
    std::mutex mu;
    uint64_t tail = 0;        // queries published
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
    cudaError_t e = launch_search(s->args, s->blocks, s->tw, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_end, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "roar_server: launch");
    s->launched = true;
    ++s->launches;
    return ROAR_OK;
}

void poll_loop(roar_server *s) {
    while (!s->quit.load(std::memory_order_acquire)) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            const Clock::time_point now = Clock::now();
            for (Request &r : s->reqs) {
                if (r.complete) continue;
                while (r.checked < r.nq) {
                    const uint64_t seq = r.first + (uint64_t)r.checked;
                    const uint32_t mark = *(volatile uint32_t *)(s->done_h + (seq % (uint64_t)s->R));
                    if (mark != (uint32_t)(seq + 1)) break;
                    ++r.checked;
                    ++s->completed_q;
                }
                if (r.checked == r.nq) {
                    std::atomic_thread_fence(std::memory_order_acquire);
                    r.complete = true;
                    r.t_done = now;
                }
            }
            // Teams exit after an idle period: relaunch if work is waiting.
            if (s->completed_q < s->tail && !kernel_running(s)) launch_locked(s);
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
    cudaError_t e = host_mapped(&s->q_h, &s->q_d, R * s->d);
    if (e == cudaSuccess) e = host_mapped(&s->k_h, &s->k_d, R);
    if (e == cudaSuccess) e = host_mapped(&s->L_h, &s->L_d, R);
    if (e == cudaSuccess) e = host_mapped(&s->ids_h, &s->ids_d, R * s->k_max);
    if (e == cudaSuccess) e = host_mapped(&s->dist_h, &s->dist_d, R * s->k_max);
    if (e == cudaSuccess) e = host_mapped(&s->vis_h, &s->vis_d, R);
    if (e == cudaSuccess) e = host_mapped(&s->hops_h, &s->hops_d, R);
    if (e == cudaSuccess) e = host_mapped(&s->st_h, &s->st_d, R);
    if (e == cudaSuccess) e = host_mapped(&s->done_h, &s->done_d, R);
    if (e == cudaSuccess) e = host_mapped(&s->tail_h, &s->tail_d, 1);
    if (e == cudaSuccess) e = host_mapped(&s->stop_h, &s->stop_d, 1);
    if (e == cudaSuccess) e = cudaMalloc(&s->head_dev, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(s->head_dev, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_end, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        roar_status rc = cuda_fail(e, "roar_server_create");
        roar_server_destroy(s);
        return rc;
    }
    a.q = s->q_d;
    a.nq = (int64_t)1 << 62;
    a.k_arr = s->k_d;
    a.L_arr = s->L_d;
    a.ids = s->ids_d;
    a.dist = s->dist_d;
    a.visits = s->vis_d;
    a.hops = s->hops_d;
    a.qstatus = s->st_d;
    a.ring_tail = s->tail_d;
    a.ring_head = s->head_dev;
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
    const uint64_t first = s->tail;
    for (int32_t i = 0; i < nq; ++i) {
        const size_t slot = (size_t)((first + (uint64_t)i) % (uint64_t)s->R);
        std::memcpy(s->q_h + slot * s->d, q_host + (size_t)i * s->d, (size_t)s->d * 4);
        s->k_h[slot] = k;
        s->L_h[slot] = L;
    }
    std::atomic_thread_fence(std::memory_order_release);
    s->tail = first + (uint64_t)nq;
    *(volatile unsigned long long *)s->tail_h = s->tail;  // publish
    std::atomic_thread_fence(std::memory_order_seq_cst);
    Request r;
    r.first = first;
    r.nq = nq;
    r.k = k;
    r.charge = charge;
    s->inflight += charge;
    r.t_submit = Clock::now();
    s->reqs.push_back(r);
    *request_id = first;
    if (!kernel_running(s)) return launch_locked(s);
    return ROAR_OK;
}

extern "C" roar_status roar_server_poll(roar_server *s, uint64_t request_id, int32_t timeout_ms,
                                        uint32_t *ids, float *dist, uint32_t *visits, int32_t *qstatus,
                                        double *latency_s) {
    if (!s || timeout_ms < 0) return ROAR_EINVAL;
    const Clock::time_point deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            Request *r = nullptr;
            for (Request &x : s->reqs)
                if (x.first == request_id && !x.released) r = &x;
            if (!r) {
                set_error("roar_server_poll: unknown or already released request");
                return ROAR_EINVAL;
            }
            if (r->complete) {
                for (int32_t i = 0; i < r->nq; ++i) {
                    const size_t slot = (size_t)((r->first + (uint64_t)i) % (uint64_t)s->R);
                    if (ids) std::memcpy(ids + (size_t)i * r->k, s->ids_h + slot * s->k_max, (size_t)r->k * 4);
                    if (dist) std::memcpy(dist + (size_t)i * r->k, s->dist_h + slot * s->k_max, (size_t)r->k * 4);
                    if (visits) visits[i] = s->vis_h[slot];
                    if (qstatus) qstatus[i] = s->st_h[slot];
                }
                if (latency_s)
                    *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
                r->released = true;
                s->inflight -= r->charge;
                // Slots free up in ring order.
                while (!s->reqs.empty() && s->reqs.front().released) {
                    s->released = s->reqs.front().first + (uint64_t)s->reqs.front().nq;
                    s->reqs.pop_front();
                }
                return ROAR_OK;
            }
        }
        if (Clock::now() >= deadline) return ROAR_ETIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
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
    if (s->stop_h) {
        *(volatile int *)s->stop_h = 1;
        std::atomic_thread_fence(std::memory_order_seq_cst);
    }
    if (s->poller.joinable()) {
        s->quit.store(true, std::memory_order_release);
        s->poller.join();
    }
    if (s->stream) cudaStreamSynchronize(s->stream);  // teams exit at their next poll
    if (s->ev_end) cudaEventDestroy(s->ev_end);
    if (s->stream) cudaStreamDestroy(s->stream);
    cudaFree(s->head_dev);
    cudaFreeHost(s->q_h);
    cudaFreeHost(s->k_h);
    cudaFreeHost(s->L_h);
    cudaFreeHost(s->ids_h);
    cudaFreeHost(s->dist_h);
    cudaFreeHost(s->vis_h);
    cudaFreeHost(s->hops_h);
    cudaFreeHost(s->st_h);
    cudaFreeHost(s->done_h);
    cudaFreeHost(s->tail_h);
    cudaFreeHost(s->stop_h);
    delete s;
}
