// roar_search_noalloc: the FP32 beam search for callers that cannot allocate
// device memory (see include/roargraph.h). All of its scratch (the query work
// counter, one visited bitmap and one visit log per resident warp) lives in
// one fixed array compiled into the library, so the call needs no handle and
// makes no allocation; it launches the same kernel as roar_search.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "roar_internal.cuh"

namespace roar {
roar_status cuda_fail(cudaError_t e, const char *what);
void set_error(const char *msg);
bool aligned(const void *p, size_t a);
}  // namespace roar

using namespace roar;

namespace {

// Fixed scratch: 64 MiB on every device that loads the library, kept until exit.
constexpr size_t kScratchBytes = (size_t)ROAR_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices];  // device address of g_scratch, per device (set up once)
int g_num_sms[kMaxDevices];

// Once per device, with that device current: look up the array's device
// address (host code cannot use the symbol itself as a pointer).
roar_status device_setup(int dev, void **addr, int *sms) {
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("roar_search_noalloc: device ordinal out of range");
        return ROAR_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "roar_search_noalloc: cudaGetSymbolAddress");
        int s = 0;
        e = cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "roar_search_noalloc: device attribute");
        g_num_sms[dev] = s;
        g_scratch_addr[dev] = p;
    }
    *addr = g_scratch_addr[dev];
    *sms = g_num_sms[dev];
    return ROAR_OK;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" roar_status roar_search_noalloc(int64_t n, int32_t d, const float *base_f32,
                                           const uint32_t *adj, int32_t rmax, uint32_t entry,
                                           uint32_t max_visits, const float *queries, int64_t nq,
                                           int32_t k, int32_t L, uint32_t *ids, float *dist,
                                           uint32_t *visits, uint32_t *hops, int32_t *qstatus,
                                           void *stream) {
    if (n < 1 || n >= (int64_t)kIdMask || d < 4 || d > 1024 || d % 4 != 0 || !base_f32 || !adj ||
        rmax < 1 || rmax > ROAR_MAX_RMAX || (int64_t)entry >= n || nq < 0 || k < 1 || L < k ||
        L > ROAR_MAX_L || max_visits > (1u << 24)) {
        set_error("roar_search_noalloc: bad size, pointer, entry, k or L");
        return ROAR_EINVAL;
    }
    if (nq == 0) return ROAR_OK;
    if (nq >= (int64_t)1 << 31 || !queries || !ids || !dist || !aligned(queries, 16) ||
        !aligned(base_f32, 16) || !aligned(adj, 4)) {
        set_error("roar_search_noalloc: bad query, base or output pointer");
        return ROAR_EINVAL;
    }
    if (max_visits == 0) max_visits = 16384u;
    // Scratch layout: [work counter][bitmap per slot][visit log per slot].
    const int64_t words = (n + 31) / 32;
    const int32_t log_cap = (int32_t)max_visits + ROAR_MAX_RMAX;
    const size_t per_slot = (size_t)words * 4 + (size_t)log_cap * 4;
    const size_t head = 256;
    // The logs start on a 256-byte boundary after the bitmaps: keep 256 bytes
    // for that padding, so every slot count up to slots_fit fits the array.
    const int64_t slots_fit = (int64_t)((kScratchBytes - head - 256) / per_slot);
    if (slots_fit < kWarpsPerBlock) {
        set_error("roar_search_noalloc: n or max_visits too large for the fixed 64 MiB scratch "
                  "(needs 4 * (ceil(n/32) + max_visits + 128) bytes per warp, 4 warps at least, "
                  "within 64 MiB - 512 bytes)");
        return ROAR_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "roar_search_noalloc: cudaGetDevice");
    void *base = nullptr;
    int sms = 0;
    roar_status st = device_setup(dev, &base, &sms);
    if (st != ROAR_OK) return st;

    SearchArgs a;
    std::memset(&a, 0, sizeof a);
    a.trav = base_f32;
    a.base32 = base_f32;
    a.adj = adj;
    a.n = n;
    a.d = d;
    a.rmax = rmax;
    a.entry = entry;
    a.dtype = ROAR_F32;
    a.lcap = (L + 31) / 32 * 32;
    a.max_visits = max_visits;
    a.hash_log2 = hash_log2_for(L);
    const int bps = search_blocks_per_sm(ROAR_F32, d, rmax, a.lcap, a.hash_log2, 1);
    if (bps <= 0) {
        set_error("roar_search_noalloc: this L does not fit in shared memory");
        return ROAR_EINVAL;
    }
    const int64_t want = (nq + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int64_t blocks = std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>(want, (int64_t)bps * sms), slots_fit / kWarpsPerBlock));
    const int64_t slots = blocks * kWarpsPerBlock;
    unsigned char *p = static_cast<unsigned char *>(base);
    a.work = reinterpret_cast<unsigned int *>(p);
    a.vbits = reinterpret_cast<uint32_t *>(p + head);
    a.vbits_words = words;
    a.vlog = reinterpret_cast<uint32_t *>(p + head + up256((size_t)slots * words * 4));
    a.vlog_cap = log_cap;
    if ((size_t)(reinterpret_cast<unsigned char *>(a.vlog) - p) + (size_t)slots * log_cap * 4 > kScratchBytes) {
        set_error("roar_search_noalloc: scratch layout overflow");
        return ROAR_EINVAL;
    }
    a.q = queries;
    a.nq = nq;
    a.k = k;
    a.L = L;
    a.ids = ids;
    a.dist = dist;
    a.visits = visits;
    a.hops = hops;
    a.qstatus = qstatus;
    cudaStream_t s = (cudaStream_t)stream;
    // The array keeps whatever the previous call left: the bitmaps must start
    // all-zero (the work counter is reset by the launch itself).
    e = cudaMemsetAsync(a.vbits, 0, (size_t)slots * words * 4, s);
    if (e != cudaSuccess) return cuda_fail(e, "roar_search_noalloc: clear");
    e = launch_search(a, (int)blocks, 1, s);
    if (e != cudaSuccess) return cuda_fail(e, "roar_search_noalloc launch");
    return ROAR_OK;
}
