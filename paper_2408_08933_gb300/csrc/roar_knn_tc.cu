// Tensor-core scores with a fused running top-C (the kNN step of the index
// construction, Sec. 4.2.1): S = T . X^T in BF16 with FP32 accumulation on the
// 5th-generation tensor cores, never written to memory.
//
// One CTA owns 128 or 256 rows of T and keeps them resident in shared memory;
// it sweeps all rows of X in tiles of 256 or 128 (the MMA's N). With 256 rows
// (d <= 256) the two 128-row halves (the MMA's M is 128) share each X tile,
// which halves the X bytes every score needs from L2. Warp roles:
// two producer warps stage 64-wide K chunks of X through a ring of up to four
// shared-memory stages (cp.async with zero fill past n and d) in the canonical
// no-swizzle K-major layout (8 x 16-byte core matrices, K-adjacent ones 128 B
// apart, 8-row groups 1024 B apart); one thread issues tcgen05.mma (kind::f16,
// BF16 x BF16 -> FP32) into one of two 256-column TMEM accumulators, so the
// next tile is computed while the last is read; four epilogue warps read their
// 32 TMEM lanes each (one row per thread) with tcgen05.ld. Per row a running
// threshold filters the scores: a column enters the row's candidate buffer
// only if it beats the threshold. Between tiles, a buffer that could not take
// another full tile is cut back to its best C by its whole warp (a bitwise
// search for the C-th largest key, then a ballot compaction), which raises the
// threshold. At the end each row's best C candidates are written out
// (unsorted) for the exact FP32 re-score.
//
// Every mbarrier wait is bounded (wait_ns of wall time per wait): on timeout
// the kernel sets *err, waits for its own copies and for the MMAs it has
// issued, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "roar_internal.cuh"

namespace roar {

roar_status cuda_fail(cudaError_t e, const char *what);

namespace {

constexpr int kTM = 128;           // T rows per MMA (its M); a CTA holds kMH such halves
constexpr int kKC = 64;            // K elements per staged chunk (128 bytes per row)
constexpr int kProducers = 64;     // warps 0-1 stage operands
constexpr int kMmaWarp = 2;        // lane 0 issues the MMAs; the warp owns TMEM
constexpr int kMaxStages = 8;
constexpr int kCap = 1024;         // candidate buffer entries per row
constexpr uint64_t kDrainNs = 2000000000ull;  // bound of the final wait for issued MMAs
constexpr int kTmemCols = 512;     // 2 buffers x kMH halves x (256 / kMH) columns
constexpr uint32_t kChunkA = kTM * kKC * 2;   // 16 KB: one half's 64-wide K chunk
constexpr unsigned kFull = 0xFFFFFFFFu;

// X rows per tile (the MMA's N), threads and B chunk bytes for kMH halves.
template <int kMH>
struct KnnShape {
    static constexpr int TN = 256 / kMH;
    static constexpr int threads = (3 + 4 * kMH) * 32;
    static constexpr uint32_t chunkB = (uint32_t)TN * kKC * 2;
    // Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
    // (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
    // M >> 4 at bit 24.
    static constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                                      ((uint32_t)(kTM >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start, leading (K) and stride (8-row group)
// byte offsets (all >> 4), descriptor version 1 (bit 46), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// The same for the 128-byte-swizzled K-major layout TMA writes: rows of 128
// bytes (64 BF16 of K), the 16-byte pieces of row r at piece ^ (r % 8),
// 8-row atoms 1024 bytes apart (stride offset); the atoms are 1024-byte
// aligned (base offset 0). A K step of 16 elements advances the start by 32
// bytes inside the atom. Swizzle mode 2 (128-byte) in bits 61-63.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    return smem_desc(saddr, 16, 1024) | ((uint64_t)2 << 61);
}

// Arm a barrier for `bytes` of asynchronous copies (one arrival).
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// TMA: the box at (x = column, y = row) of the 2-D tensor map to shared
// memory; completion counted in bytes on `bar`.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int32_t x, int32_t y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity: gives up (and raises the
// CTA's abort flag) after wait_ns of wall time, or as soon as another role
// aborted. wait_ns == 0 gives up as soon as the phase is found incomplete
// (a test setting: it makes the timeout path run without any fault).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort, uint64_t wait_ns) {
    if (wait_ns == 0) {
        if (mbar_test(bar, parity)) return true;
        *abort = 1;
        return false;
    }
    uint64_t deadline = 0;
    for (uint32_t i = 0;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if (*abort) return false;
        if ((i & 63) == 0) {
            const uint64_t now = global_ns();
            if (deadline == 0) deadline = now + wait_ns;
            else if (now > deadline) {
                *abort = 1;
                return false;
            }
        }
    }
}

// Bounded wait that ignores the abort flag: the final wait for the MMAs this
// thread issued (they always complete; the bound only keeps the wait finite).
__device__ __forceinline__ bool mbar_drain(uint64_t *bar, uint32_t parity) {
    uint64_t deadline = 0;
    for (uint32_t i = 0;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 63) == 0) {
            const uint64_t now = global_ns();
            if (deadline == 0) deadline = now + kDrainNs;
            else if (now > deadline) return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// The barrier's phase completes once this thread's earlier cp.async copies land.
__device__ __forceinline__ void cp_async_arrive(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// Issue a load of 32 consecutive FP32 columns of this thread's TMEM lane; the
// registers are valid only after tc_wait_ld.
__device__ __forceinline__ void tc_ld32_issue(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
}

// Wait for this thread's TMEM loads. The registers of the loads pass through
// the statement, so no use of them can be scheduled before the wait.
__device__ __forceinline__ void tc_wait_ld(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// Orders later uses of `r` after the preceding (volatile) wait.
__device__ __forceinline__ void reg_after_wait(uint32_t (&r)[32]) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}

// Order-preserving map of a finite float to uint32 (larger float, larger key).
__device__ __forceinline__ uint32_t f2key(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key2f(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// The whole warp cuts one row's buffer (scores s, ids c, m <= kCap entries) to
// its best `keep` in place and returns the keep-th best score. The keep-th
// largest key is found bit by bit from the top (the largest t with at least
// `keep` keys >= t); every key above t is kept, then keys equal to t in buffer
// order until `keep` are kept. Must be called by all 32 lanes with the same
// arguments, after the lane that filled the buffer has passed a __syncwarp.
__device__ float warp_cut(float *s, uint32_t *c, int m, int keep, int lane) {
    constexpr int kPer = kCap / 32;
    uint32_t key[kPer], id[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int j = i * 32 + lane;
        key[i] = j < m ? f2key(s[j]) : 0u;
        id[i] = j < m ? c[j] : 0u;
    }
    uint32_t t = 0;
    for (int bit = 31; bit >= 0; --bit) {
        const uint32_t cand = t | (1u << bit);
        uint32_t cnt = 0;
#pragma unroll
        for (int i = 0; i < kPer; ++i) cnt += key[i] >= cand ? 1u : 0u;
        if ((int)__reduce_add_sync(kFull, cnt) >= keep) t = cand;
    }
    __syncwarp();  // every lane has read the buffer before it is rewritten
    const uint32_t lt = (1u << lane) - 1u;
    int pos = 0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const bool take = i * 32 + lane < m && key[i] > t;
        const uint32_t b = __ballot_sync(kFull, take);
        if (take) {
            const int p = pos + __popc(b & lt);
            s[p] = key2f(key[i]);
            c[p] = id[i];
        }
        pos += __popc(b);
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const bool tie = i * 32 + lane < m && key[i] == t;
        const uint32_t b = __ballot_sync(kFull, tie);
        const int p = pos + __popc(b & lt);
        if (tie && p < keep) {
            s[p] = key2f(key[i]);
            c[p] = id[i];
        }
        pos += __popc(b);
    }
    __syncwarp();
    return key2f(t);
}

// Stage one 64-wide K chunk of `rows` rows starting at global row r0 into the
// core-matrix layout at `dst` (zero fill past nrows and past d); thread `tid`
// of `nthr` takes every nthr-th 16-byte piece.
__device__ __forceinline__ void stage_chunk(uint32_t dst, const __nv_bfloat16 *src, int64_t r0, int rows,
                                            int64_t nrows, int d, int k0, int tid, int nthr) {
    const int pieces = rows * (kKC / 8);
    for (int p = tid; p < pieces; p += nthr) {
        const int row = p >> 3, kg = p & 7;
        const int64_t gr = r0 + row;
        const int k = k0 + kg * 8;
        const bool ok = gr < nrows && k < d;
        const __nv_bfloat16 *g = ok ? src + gr * d + k : src;
        const uint32_t off = (uint32_t)(((row >> 3) * 8 + kg) * 128 + (row & 7) * 16);
        cp_async16(dst + off, g, ok ? 16u : 0u);
    }
}

// Warp roles: 0-1 stage operands (cp.async, completion on per-stage "full"
// barriers), 2 issues the MMAs (lane 0; stage freed through "empty" barriers
// by tcgen05.commit) and owns TMEM, 3 .. 3 + 4 kMH - 1 read the two
// alternating accumulators while the next tile is computed: warp w reads TMEM
// lanes 32 * (w % 4) .. + 31 of half (w - 3) / 4, one T row per thread.
// kTma: operands staged by TMA (one thread issues 2-D tensor-map copies into
// the 128-byte-swizzled layout, completion counted in bytes on the "full"
// barriers) instead of the two cp.async producer warps and the no-swizzle
// layout. kMH: 128-row halves of T per CTA (2 needs kTma).
template <bool kTma, int kMH>
__global__ void __launch_bounds__(KnnShape<kMH>::threads, 1)
knn_tc_kernel(const __nv_bfloat16 *__restrict__ T, int64_t nt, const __nv_bfloat16 *__restrict__ X,
              int64_t n, int d, int stages, int C, float *__restrict__ buf_s,
              uint32_t *__restrict__ buf_i, uint32_t *__restrict__ out_i, int *__restrict__ err,
              uint64_t wait_ns, const __grid_constant__ CUtensorMap tmA,
              const __grid_constant__ CUtensorMap tmB) {
    static_assert(kTma || kMH == 1, "the cp.async producers stage one half");
    constexpr int kTN = KnnShape<kMH>::TN;
    constexpr uint32_t kChunkB = KnnShape<kMH>::chunkB;
    constexpr uint32_t kIdesc = KnnShape<kMH>::idesc;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], acc_full[2], acc_empty[2], a_full, drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    volatile int *abort_v = &abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nkc = (d + kKC - 1) / kKC;
    // TMA's 128-byte swizzle repeats every 1024 bytes: start the operands there.
    const uint32_t a_base = kTma ? ((smem_addr(smem) + 1023u) & ~1023u) : smem_addr(smem);
    const uint32_t b_base = a_base + (uint32_t)(nkc * kMH) * kChunkA;
    const int64_t m0 = (int64_t)blockIdx.x * (kTM * kMH);
    const int64_t ntiles = (n + kTN - 1) / kTN;
    const int64_t nchunks = ntiles * nkc;


    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full_bar[s], kTma ? 1 : kProducers);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4 * 32 * kMH);
        }
        mbar_init(&a_full, kTma ? 1 : kProducers);
        mbar_init(&drain_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (kTma && warp < 2) {
        // ---- producer: one thread issues every TMA copy ----
        if (warp == 0 && lane == 0) {
            // Per stage: armed at least once, and the parity of the last phase armed.
            bool armed[kMaxStages];
            uint32_t last_par[kMaxStages];
            for (int i = 0; i < kMaxStages; ++i) {
                armed[i] = false;
                last_par[i] = 0;
            }
            mbar_expect_tx(&a_full, (uint32_t)(nkc * kMH) * kChunkA);
            for (int c = 0; c < nkc; ++c)
                for (int h = 0; h < kMH; ++h)
                    tma_load_2d(a_base + (uint32_t)(c * kMH + h) * kChunkA, &tmA, c * kKC, (int32_t)(m0 + kTM * h),
                                &a_full);
            // Chunk g is K chunk c of tile t in stage s, the stage's use number
            // `wrap`: counters, not divisions (64-bit division is slow).
            int s = 0, c = 0;
            uint32_t wrap = 0;
            int64_t t = 0;
            for (int64_t g = 0; g < nchunks; ++g) {
                if (wrap > 0 && !mbar_wait(&empty_bar[s], (wrap - 1) & 1, abort_v, wait_ns)) break;
                mbar_expect_tx(&full_bar[s], kChunkB);
                tma_load_2d(b_base + (uint32_t)s * kChunkB, &tmB, c * kKC, (int32_t)(t * kTN), &full_bar[s]);
                armed[s] = true;
                last_par[s] = wrap & 1;
                if (++c == nkc) {
                    c = 0;
                    ++t;
                }
                if (++s == stages) {
                    s = 0;
                    ++wrap;
                }
            }
            // No copy may still be landing when the CTA exits (after an abort
            // some armed stages are never consumed): wait, bounded, for the
            // last phase armed on every barrier.
            bool drained = mbar_drain(&a_full, 0);
            for (int i = 0; i < stages; ++i)
                if (armed[i]) drained = mbar_drain(&full_bar[i], last_par[i]) && drained;
            if (!drained) *abort_v = 1;
        }
        __syncwarp();
    } else if (warp < 2) {
        // ---- producers ----
        for (int c = 0; c < nkc; ++c) stage_chunk(a_base + (uint32_t)c * kChunkA, T, m0, kTM, nt, d, c * kKC, tid, kProducers);
        cp_async_arrive(&a_full);
        int s = 0, c = 0;
        uint32_t wrap = 0;
        int64_t t = 0;
        for (int64_t g = 0; g < nchunks; ++g) {
            if (wrap > 0 && !mbar_wait(&empty_bar[s], (wrap - 1) & 1, abort_v, wait_ns)) break;
            stage_chunk(b_base + (uint32_t)s * kChunkB, X, t * kTN, kTN, n, d, c * kKC, tid, kProducers);
            cp_async_arrive(&full_bar[s]);
            if (++c == nkc) {
                c = 0;
                ++t;
            }
            if (++s == stages) {
                s = 0;
                ++wrap;
            }
        }
        cp_async_wait<0>();
    } else if (warp == kMmaWarp) {
        // ---- MMA issue ----
        if (lane == 0) {
            bool issued = false;
            if (mbar_wait(&a_full, 0, abort_v, wait_ns)) {
                if (!kTma) fence_async_smem();  // cp.async data, written through the generic proxy, to the tensor core
                // Descriptors of the operand bases; a chunk, a half or a K step
                // moves the start address field (bytes >> 4).
                const uint64_t adesc0 = kTma ? smem_desc_sw128(a_base) : smem_desc(a_base, 128, 1024);
                const uint64_t bdesc0 = kTma ? smem_desc_sw128(b_base) : smem_desc(b_base, 128, 1024);
                constexpr uint32_t kStep = kTma ? 32 >> 4 : 256 >> 4;   // one K step of 16
                int s = 0;
                uint32_t wrap = 0;
                bool ok = true;
                for (int64_t t = 0; t < ntiles && ok; ++t) {
                    const int b = (int)(t & 1);
                    const uint32_t ub = (uint32_t)(t >> 1);
                    if (ub > 0 && !mbar_wait(&acc_empty[b], (ub - 1) & 1, abort_v, wait_ns)) break;
                    tc_fence_after();
                    for (int c = 0; c < nkc; ++c) {
                        if (!mbar_wait(&full_bar[s], wrap & 1, abort_v, wait_ns)) {
                            ok = false;
                            break;
                        }
                        if (!kTma) fence_async_smem();
                        tc_fence_after();
                        const uint64_t bd0 = bdesc0 + (((uint32_t)s * kChunkB) >> 4);
                        const uint64_t ad0 = adesc0 + (((uint32_t)(c * kMH) * kChunkA) >> 4);
#pragma unroll
                        for (int ks = 0; ks < kKC / 16; ++ks) {
#pragma unroll
                            for (int h = 0; h < kMH; ++h)
                                tc_mma(tmem + (uint32_t)((b * kMH + h) * kTN), ad0 + h * (kChunkA >> 4) + ks * kStep,
                                       bd0 + ks * kStep, kIdesc, (c > 0 || ks > 0) ? 1u : 0u);
                        }
                        issued = true;
                        tc_commit(&empty_bar[s]);
                        if (++s == stages) {
                            s = 0;
                            ++wrap;
                        }
                    }
                    if (ok) tc_commit(&acc_full[b]);
                }
            }
            // Every MMA this thread issued has finished (it may still be
            // writing TMEM and reading shared memory after an abort) before
            // the CTA frees its TMEM and exits.
            if (issued) {
                tc_commit(&drain_bar);
                if (!mbar_drain(&drain_bar, 0)) *abort_v = 1;
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: filter each tile's scores into the row buffers ----
        // A buffer is cut back to its best C (by the whole warp) between tiles,
        // once it could not take another full tile; the cut raises the row's
        // threshold. The accumulator is released before the cuts run.
        const int q = warp & 3;
        const int half = (warp - 3) >> 2;
        const int64_t wrow0 = m0 + kTM * half + 32 * q;
        const int64_t row = wrow0 + lane;
        const bool row_ok = row < nt;
        float *rs = buf_s + (row_ok ? row : 0) * (int64_t)kCap;
        uint32_t *ri = buf_i + (row_ok ? row : 0) * (int64_t)kCap;
        int cnt = 0;
        float thr = -__int_as_float(0x7f800000);
        bool done = true;
        for (int64_t t = 0; t < ntiles; ++t) {
            const int b = (int)(t & 1);
            // The warp leaves together: the TMEM loads below are warp-collective.
            if (!__all_sync(kFull, mbar_wait(&acc_full[b], (uint32_t)(t >> 1) & 1, abort_v, wait_ns))) {
                done = false;
                break;
            }
            tc_fence_after();
            const int64_t n0 = t * kTN;
            const int lim = (int)((n - n0) < kTN ? (n - n0) : kTN);
            // kGW columns per TMEM read (loads in flight together, one wait):
            // 128 with two halves (two epilogue warps per SM sub-partition),
            // 64 with one (measured faster on GB300 for each shape).
            constexpr int kGW = kMH == 2 ? 128 : 64;
#pragma unroll 1
            for (int cb = 0; cb < kTN; cb += kGW) {
                uint32_t r0[32], r1[32], r2[32], r3[32];
                const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((b * kMH + half) * kTN + cb);
                tc_ld32_issue(taddr, r0);
                tc_ld32_issue(taddr + 32, r1);
                if constexpr (kGW == 128) {
                    tc_ld32_issue(taddr + 64, r2);
                    tc_ld32_issue(taddr + 96, r3);
                }
                tc_wait_ld(r0);
                reg_after_wait(r1);
                if constexpr (kGW == 128) {
                    reg_after_wait(r2);
                    reg_after_wait(r3);
                }
                if (!row_ok) continue;
                // Most column groups hold nothing above the row's threshold
                // once the first tiles have set it: test their maximum first.
                float mp[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    mp[i] = fmaxf(__uint_as_float(r0[i]), __uint_as_float(r1[i]));
                    if constexpr (kGW == 128)
                        mp[i] = fmaxf(mp[i], fmaxf(__uint_as_float(r2[i]), __uint_as_float(r3[i])));
                }
#pragma unroll
                for (int i = 8; i < 32; ++i) {
                    mp[i & 7] = fmaxf(mp[i & 7], fmaxf(__uint_as_float(r0[i]), __uint_as_float(r1[i])));
                    if constexpr (kGW == 128)
                        mp[i & 7] = fmaxf(mp[i & 7], fmaxf(__uint_as_float(r2[i]), __uint_as_float(r3[i])));
                }
                const float m = fmaxf(fmaxf(fmaxf(mp[0], mp[1]), fmaxf(mp[2], mp[3])),
                                      fmaxf(fmaxf(mp[4], mp[5]), fmaxf(mp[6], mp[7])));
                if (!(m > thr)) continue;
                auto take = [&](const uint32_t (&rr)[32], int c0) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const float v = __uint_as_float(rr[i]);
                        if (v > thr && c0 + i < lim) {
                            rs[cnt] = v;
                            ri[cnt] = (uint32_t)(n0 + c0 + i);
                            ++cnt;
                        }
                    }
                };
                take(r0, cb);
                take(r1, cb + 32);
                if constexpr (kGW == 128) {
                    take(r2, cb + 64);
                    take(r3, cb + 96);
                }
            }
            tc_fence_before();
            mbar_arrive(&acc_empty[b]);
            __syncwarp();
            uint32_t full = __ballot_sync(kFull, row_ok && cnt > kCap - kTN);
            while (full) {
                const int src = __ffs(full) - 1;
                full &= full - 1;
                const int m = __shfl_sync(kFull, cnt, src);
                const float th = warp_cut(buf_s + (wrow0 + src) * kCap, buf_i + (wrow0 + src) * kCap, m, C, lane);
                if (lane == src) {
                    thr = th;
                    cnt = C;
                }
            }
        }
        if (__all_sync(kFull, done && !*abort_v)) {
            uint32_t over = __ballot_sync(kFull, row_ok && cnt > C);
            while (over) {
                const int src = __ffs(over) - 1;
                over &= over - 1;
                const int m = __shfl_sync(kFull, cnt, src);
                warp_cut(buf_s + (wrow0 + src) * kCap, buf_i + (wrow0 + src) * kCap, m, C, lane);
                if (lane == src) cnt = C;
            }
            if (row_ok)
                for (int j = 0; j < C; ++j) out_i[row * (int64_t)C + j] = j < cnt ? ri[j] : 0xFFFFFFFFu;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_v && tid == 0) atomicExch(err, 1);
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// Halves of T per CTA: two while both halves' rows fit beside four stages,
// unless one-half CTAs finish nt rows sooner. Every CTA sweeps all of X, a
// two-half CTA in about twice the time (measured 0.55 of it for one half);
// so a launch takes ceil(nt / (sms * 256)) two-half sweeps or
// ceil(nt / (sms * 128)) one-half ones (a 14,336-row remainder: one sweep of
// either, the one-half one the shorter).
int knn_tc_halves(int d, bool tma, int64_t nt, int sms) {
    const int nkc = (d + kKC - 1) / kKC;
    if (!tma || nkc > 4) return 1;
    if (nt <= 0 || sms <= 0) return 2;
    const int64_t w2 = (nt + (int64_t)sms * 2 * kTM - 1) / ((int64_t)sms * 2 * kTM);
    const int64_t w1 = (nt + (int64_t)sms * kTM - 1) / ((int64_t)sms * kTM);
    return 100 * w2 <= 55 * w1 ? 2 : 1;
}

int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 1;
    cudaGetLastError();
    return sms;
}

int knn_tc_stages(int d, int mh) {
    const int nkc = (d + kKC - 1) / kKC;
    const int budget = 225 * 1024 - nkc * mh * (int)kChunkA;
    int s = budget / (int)(mh == 2 ? KnnShape<2>::chunkB : KnnShape<1>::chunkB);
    return s > kMaxStages ? kMaxStages : s;
}

}  // namespace

size_t knn_tc_smem_bytes(int d, int mh) {
    const int nkc = (d + kKC - 1) / kKC;
    const size_t need = (size_t)nkc * mh * kChunkA +
                        (size_t)knn_tc_stages(d, mh) * (mh == 2 ? KnnShape<2>::chunkB : KnnShape<1>::chunkB) + 1024;
    return need < 120 * 1024 ? 120 * 1024 : need;  // one CTA per SM: it holds all 512 TMEM columns
}

namespace {

// cuTensorMapEncodeTiled, looked up through the runtime (no link to the
// driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// A BF16 matrix [rows][d] (row-major, d % 8 == 0 so rows are 16-byte multiples)
// read in boxes of 64 columns x box_rows rows with the 128-byte swizzle; reads
// past the last row or column return zeros.
bool make_map(CUtensorMap *m, const __nv_bfloat16 *base, int64_t rows, int d, int box_rows) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)d * 2u};
    const cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Operand staging of the kNN kernel: TMA (1) or the cp.async producer warps
// (0). ROAR_KNN_TMA in the environment overrides the default.
#ifndef ROAR_KNN_TMA_DEFAULT
#define ROAR_KNN_TMA_DEFAULT 1
#endif
static int knn_env_int(const char *name, int dflt) {
    const char *e = std::getenv(name);
    return e ? std::atoi(e) : dflt;
}
static bool knn_use_tma() {
    static const bool use = []() {
        const char *e = std::getenv("ROAR_KNN_TMA");
        return e ? std::atoi(e) != 0 : ROAR_KNN_TMA_DEFAULT != 0;
    }();
    return use;
}

// T rows one full wave of the kNN kernel covers (one CTA per SM).
int64_t knn_tc_wave_rows(int d) {
    const int sms = device_sms();
    const bool want = knn_use_tma() && (d % 8) == 0;
    const int mh = knn_env_int("ROAR_KNN_HALVES", 0) == 1 ? 1 : knn_tc_halves(d, want, 0, sms);   // whole waves of the wider shape
    return (int64_t)sms * kTM * mh;
}

// Candidates (best C per row, unsorted, 0xFFFFFFFF padded) of nt rows of T16
// against X16 into cand [nt][C]; buf_s/buf_i are [nt][cap] scratch.
cudaError_t knn_tc_launch(const __nv_bfloat16 *T16, int64_t nt, const __nv_bfloat16 *X16, int64_t n, int d,
                          int C, int cap, float *buf_s, uint32_t *buf_i, uint32_t *cand, int *err,
                          uint64_t wait_ns, cudaStream_t s) {
    alignas(64) CUtensorMap tmA, tmB;
    std::memset(&tmA, 0, sizeof tmA);
    std::memset(&tmB, 0, sizeof tmB);
    const bool want = knn_use_tma() && (d % 8) == 0;
    int mh = knn_tc_halves(d, want, nt, device_sms());
    // ROAR_KNN_HALVES=1 or 2 in the environment (read at every call) forces
    // the shape where it can run; tests use it to cover both.
    const int mh_env = knn_env_int("ROAR_KNN_HALVES", 0);
    if (mh_env == 1 || (mh_env == 2 && knn_tc_halves(d, want, 0, 1) == 2)) mh = mh_env;

    const bool tma = want && make_map(&tmA, T16, nt, d, kTM) && make_map(&tmB, X16, n, d, 256 / mh);
    if (!tma) mh = 1;   // tensor maps refused: the cp.async producers stage one half
    const int tn = 256 / mh;
    const int stages = knn_tc_stages(d, mh);
    // A cut must leave room for a whole tile: C + tn <= kCap.
    if (stages < 2 || cap != kCap || C < 1 || C + tn > kCap) return cudaErrorInvalidValue;
    const size_t smem = knn_tc_smem_bytes(d, mh);
    const int64_t blocks = (nt + kTM * mh - 1) / (kTM * mh);
    cudaError_t e;
    if (mh == 2) {
        e = cudaFuncSetAttribute(knn_tc_kernel<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        knn_tc_kernel<true, 2><<<(unsigned)blocks, KnnShape<2>::threads, smem, s>>>(
            T16, nt, X16, n, d, stages, C, buf_s, buf_i, cand, err, wait_ns, tmA, tmB);
    } else if (tma) {
        e = cudaFuncSetAttribute(knn_tc_kernel<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        knn_tc_kernel<true, 1><<<(unsigned)blocks, KnnShape<1>::threads, smem, s>>>(
            T16, nt, X16, n, d, stages, C, buf_s, buf_i, cand, err, wait_ns, tmA, tmB);
    } else {
        e = cudaFuncSetAttribute(knn_tc_kernel<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        knn_tc_kernel<false, 1><<<(unsigned)blocks, KnnShape<1>::threads, smem, s>>>(
            T16, nt, X16, n, d, stages, C, buf_s, buf_i, cand, err, wait_ns, tmA, tmB);
    }
    return cudaGetLastError();
}

}  // namespace roar
