#pragma once
// Batched beam search over a RoarGraph index (Sec. 4.3): the kernel template.
// Included once per traversal type (roar_search_{f32,bf16,fp8}.cu).
//
// Per warp, in shared memory: the size-L candidate pool sorted by
// (distance, id) with an "expanded" bit in each id, the new candidates of the
// current hop, and optionally a small exact visited table (open addressing,
// linear probing). Once that table would pass half load, or when it is
// disabled, the visited set continues in a per-warp bitmap in global memory
// (one bit per base row, set with one atomicOr round trip); every id set
// there is appended to a per-warp log, and at the end of the query the log
// clears exactly those words, so the bitmap is all-zero between queries.
//
// Each hop: pick the first unexpanded pool entry, read its adjacency row
// (coalesced, one id per lane), test-and-insert the neighbours into the
// visited set, gather the new rows and score them with a warp-cooperative dot
// product in one fixed order, then merge the scored candidates into the pool
// in place. The fixed order (element i to lane (i >> 2) & 31, fmaf per lane in
// increasing i, then s += shfl_xor(s, o) for o = 16, 8, 4, 2, 1) is exactly
// what a float4 load per lane produces, and makes every distance, and hence
// the whole trajectory, independent of the batch and of the launch shape.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "roar_internal.cuh"

namespace roar {

// Global nanosecond timer (the serving loop's idle clock).
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ bool less_entry(float da, uint32_t ia, float db, uint32_t ib) {
    return da < db || (da == db && ia < ib);
}

// 16 bytes global -> shared, asynchronous, cached in L2 only.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
// 4 or 8 bytes global -> shared, asynchronous (cached in L1 and L2).
template <int N>
__device__ __forceinline__ void cp_async_small(void *smem_dst, const void *gsrc) {
    static_assert(N == 4 || N == 8, "cp.async.ca sizes");
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gsrc), "n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ float4 ld_stream_f4(const float4 *p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint2 ld_stream_u2(const uint2 *p) {
    uint2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];"
                 : "=r"(v.x), "=r"(v.y)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint32_t ld_stream_u1(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Ask L2 for rows ids_s[0..cnt) of `base` (rowbytes each): every 128-byte
// line a row touches, the (row, line) pairs spread over the warp's lanes. A
// plain hint: no register holds the data and nothing waits for it, so all of
// a hop's rows are requested from DRAM at once and the batched loads that
// follow mostly hit L2. Only valid ids are passed (checked against n).
// (Measured on GB300, 1M x 200: asking L2 for every neighbour's row as soon
// as the adjacency row arrives, before the visited set filters them, was 10-50 %
// slower in every form: the extra DRAM traffic costs more than the round trip
// it saves. Only the new rows are asked for.)
#ifndef ROAR_PREFETCH_ROWS
#define ROAR_PREFETCH_ROWS 1
#endif
__device__ __forceinline__ void prefetch_rows_l2(const void *base, uint32_t rowbytes, const uint32_t *ids_s, int cnt,
                                                 int lane) {
    const uint32_t lines = ((rowbytes + 127u) >> 7) + 1u;   // a row off a 128-byte boundary touches one more
    int lg = 0;
    while ((1u << lg) < lines) ++lg;
    const int total = cnt << lg;
    for (int idx = lane; idx < total; idx += 32) {
        const uint32_t r = (uint32_t)idx >> lg, j = (uint32_t)idx & ((1u << lg) - 1u);
        if (j < lines) {
            const uint32_t off = min(j * 128u, rowbytes - 1u);
            const char *p = static_cast<const char *>(base) + (size_t)(ids_s[r] & kIdMask) * rowbytes + off;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
        }
    }
}

// Raw 4-element chunk of a row in the traversal format.
template <int DT>
struct RawChunk;
template <>
struct RawChunk<0> {
    float4 v;
};
template <>
struct RawChunk<1> {
    uint2 v;
};
template <>
struct RawChunk<2> {
    uint32_t v;
};

template <int DT>
__device__ __forceinline__ void load_chunk(RawChunk<DT> &r, const void *base, uint32_t u, int d,
                                           int ch) {
    if constexpr (DT == 0) {
        r.v = ld_stream_f4(reinterpret_cast<const float4 *>(static_cast<const float *>(base) +
                                                            (size_t)u * d) + ch);
    } else if constexpr (DT == 1) {
        r.v = ld_stream_u2(reinterpret_cast<const uint2 *>(static_cast<const uint16_t *>(base) +
                                                           (size_t)u * d) + ch);
    } else {
        r.v = ld_stream_u1(reinterpret_cast<const uint32_t *>(static_cast<const uint8_t *>(base) +
                                                              (size_t)u * d) + ch);
    }
}

template <int DT>
__device__ __forceinline__ float4 to_f4(const RawChunk<DT> &r) {
    if constexpr (DT == 0) {
        return r.v;
    } else if constexpr (DT == 1) {
        // BF16 -> FP32 is exact: the BF16 bits are the top half of the FP32 bits.
        return make_float4(__uint_as_float(r.v.x << 16), __uint_as_float(r.v.x & 0xFFFF0000u),
                           __uint_as_float(r.v.y << 16), __uint_as_float(r.v.y & 0xFFFF0000u));
    } else {
        // E4M3 -> FP16 -> FP32, both exact. Byte j of the word is element 4ch + j.
        __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(r.v & 0xFFFFu), __NV_E4M3);
        __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(r.v >> 16), __NV_E4M3);
        float2 a = __half22float2(*reinterpret_cast<__half2 *>(&lo));
        float2 b = __half22float2(*reinterpret_cast<__half2 *>(&hi));
        return make_float4(a.x, a.y, b.x, b.y);
    }
}

// Rows gathered per batch: FP32 rows about ROAR_BATCH_CHUNKS 16-byte loads in
// flight per lane (measured on GB300: 12 with 4 CTAs per SM beat 8 with 5, and
// every deeper or shallower pairing); BF16 / FP8 chunks are 8 / 4 bytes, so
// twice as many rows (at most ROAR_LOWP_MAX_ROWS) fit the same registers.
#ifndef ROAR_BATCH_CHUNKS
#define ROAR_BATCH_CHUNKS 12
#endif
#ifndef ROAR_LOWP_MAX_ROWS
#define ROAR_LOWP_MAX_ROWS 8
#endif
// The FP32 re-rank inside the BF16 / FP8 kernels gathers fewer rows per batch
// (ROAR_RERANK_CHUNKS loads per lane): those kernels run with fewer registers.
// With wide rows (ROAR_RERANK_CHUNKS_WIDE; on GB300 at 1M x 512, 8 chunks,
// i.e. 2 rows per batch, beat 16 by 3-10 %: the wider batch spilled).
#ifndef ROAR_RERANK_CHUNKS
#define ROAR_RERANK_CHUNKS 8
#endif
#ifndef ROAR_RERANK_CHUNKS_WIDE
#define ROAR_RERANK_CHUNKS_WIDE 8
#endif
template <int NCH>
__host__ __device__ constexpr int rerank_rows() {
    return NCH >= 4 ? (NCH >= ROAR_RERANK_CHUNKS_WIDE ? 1 : ROAR_RERANK_CHUNKS_WIDE / NCH)
                    : (NCH >= ROAR_RERANK_CHUNKS ? 1 : ROAR_RERANK_CHUNKS / NCH);
}
template <int DT, int NCH>
__host__ __device__ constexpr int batch_rows() {
    constexpr int f32 = NCH >= ROAR_BATCH_CHUNKS ? 1 : ROAR_BATCH_CHUNKS / NCH;
    constexpr int lowp = 2 * f32 > ROAR_LOWP_MAX_ROWS ? (f32 > ROAR_LOWP_MAX_ROWS ? f32 : ROAR_LOWP_MAX_ROWS) : 2 * f32;
    return DT == 0 ? f32 : lowp;
}

// Sums of B rows over the warp at once, in the fixed butterfly order
// (s = s + s(lane xor o) for o = 16, 8, 4, 2, 1). On entry s[b] is this
// lane's partial sum of row b. While a lane still holds several rows, each
// level keeps half of them and hands the other half to the partner lane, so
// every addition has exactly the operands of the butterfly's (a + b == b + a
// bit for bit) with fewer shuffles. On exit the lane holds the complete sum
// of row lane / reduce_stride<B>(); lanes reduce_stride<B>() apart hold
// consecutive rows, those with lane % reduce_stride<B>() == 0 write them.
template <int B>
__host__ __device__ constexpr int rows_pow2() {
    return B <= 1 ? 1 : (B <= 2 ? 2 : (B <= 4 ? 4 : (B <= 8 ? 8 : (B <= 16 ? 16 : 32))));
}
template <int B>
__host__ __device__ constexpr int reduce_stride() {
    return 32 / rows_pow2<B>();
}
template <int B>
__device__ __forceinline__ float reduce_rows(const float (&s)[B], int lane) {
    static_assert(B >= 1 && B <= 32, "1 to 32 rows");
    constexpr int P = rows_pow2<B>();
    float v[P];
#pragma unroll
    for (int j = 0; j < P; ++j) v[j] = j < B ? s[j] : 0.0f;
#pragma unroll
    for (int o = 16, R = P; R > 1; o >>= 1, R >>= 1) {
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < R / 2; ++j) {
            const float keep = hi ? v[j + R / 2] : v[j];
            const float send = hi ? v[j] : v[j + R / 2];
            v[j] = keep + __shfl_xor_sync(kFull, send, o);
        }
    }
#pragma unroll
    for (int o = 16 / P; o >= 1; o >>= 1) v[0] = v[0] + __shfl_xor_sync(kFull, v[0], o);   // (none when P = 32)
    return v[0];
}

// Distances for rows ids_s[j] (shared, expanded bit ignored), j = first,
// first + 1, ... in groups of B, groups `step` apart (one warp's share of a
// team); writes -<q, x> (times the row scale for FP8) to out_s[j].
// ahead > 0: while scoring a batch, ask L2 for this warp's batch `ahead`
// batches later (and for the first `ahead` batches up front).
template <int DT, int NCH, int B>
__device__ __forceinline__ void score_rows(const void *base, const float *scales, int d, int d4,
                                           const float4 (&qr)[NCH], const uint32_t *ids_s, int cnt,
                                           float *out_s, int lane, int first = 0, int step = B, int ahead = 0) {
    constexpr int RS = reduce_stride<B>();
    const uint32_t rowbytes = (uint32_t)d * (4u >> DT);
    if (ROAR_PREFETCH_ROWS)
        for (int a = 0; a < ahead; ++a) {
            const int p0 = first + a * step;
            if (p0 < cnt) prefetch_rows_l2(base, rowbytes, ids_s + p0, min(B, cnt - p0), lane);
        }
    const int rr = lane / RS;                          // the row this lane sums and writes
    const bool writer = (lane & (RS - 1)) == 0 && rr < B;
    for (int j0 = first; j0 < cnt; j0 += step) {
        if (ROAR_PREFETCH_ROWS && ahead > 0) {
            const int p0 = j0 + ahead * step;
            if (p0 < cnt) prefetch_rows_l2(base, rowbytes, ids_s + p0, min(B, cnt - p0), lane);
        }
        RawChunk<DT> raw[B][NCH];
        float sc = 1.0f;  // FP8: the writer of row j0 + rr holds its scale, loaded with the rows
        if constexpr (DT == 2) {
            if (scales && writer && j0 + rr < cnt) sc = __ldg(scales + (ids_s[j0 + rr] & kIdMask));
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int j = j0 + b;
            const uint32_t u = j < cnt ? (ids_s[j] & kIdMask) : 0u;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int ch = lane + 32 * c;
                if (j < cnt && ch < d4) load_chunk<DT>(raw[b][c], base, u, d, ch);
            }
        }
        float s[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            s[b] = 0.0f;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int ch = lane + 32 * c;
                if (ch < d4) {
                    const float4 x = to_f4<DT>(raw[b][c]);
                    s[b] = fmaf(qr[c].x, x.x, s[b]);
                    s[b] = fmaf(qr[c].y, x.y, s[b]);
                    s[b] = fmaf(qr[c].z, x.z, s[b]);
                    s[b] = fmaf(qr[c].w, x.w, s[b]);
                }
            }
        }
        const float mine = reduce_rows<B>(s, lane);
        __syncwarp();
        if (writer && j0 + rr < cnt) {
            if constexpr (DT == 2) {
                out_s[j0 + rr] = -(sc * mine);
            } else {
                out_s[j0 + rr] = -mine;
            }
        }
    }
    __syncwarp();
}

// Distances for rows ids_s[0..cnt) through shared memory (one warp). The
// warp copies S rows at a time, in 16-byte pieces (piece p on lane p % 32;
// for FP8 lane r also the scale of row r), into one of two buffers with
// cp.async, so the next S rows are in flight while these are scored. After
// the copies land (each lane waits for its own, then the warp synchronises)
// every lane reads its chunks (chunk c on lane c % 32, as in score_rows): the
// decode, the arithmetic and its order are score_rows' exactly. Needs
// 16-byte-aligned rows (d * element bytes a multiple of 16).
template <int DT, int NCH, int S>
__device__ __forceinline__ void score_rows_staged(const void *base, const float *scales, int d4,
                                                  const float4 (&qr)[NCH], const uint32_t *ids_s, int cnt,
                                                  float *out_s, int lane, unsigned char *stg) {
    using Chunk = decltype(RawChunk<DT>::v);
    constexpr int CB = (int)sizeof(Chunk);
    static_assert(CB == chunk_bytes(DT), "chunk size");
    const int rowbytes = d4 * CB;
    const int pieces = rowbytes >> 4;                 // <= d4 <= 32 * NCH
    unsigned char *cbuf = stg;
    float *sbuf = reinterpret_cast<float *>(stg + (size_t)2 * S * rowbytes);   // FP8 row scales
    const unsigned char *rows = static_cast<const unsigned char *>(base);
    const int nb = (cnt + S - 1) / S;
    auto issue = [&](int bi) {
        unsigned char *buf = cbuf + (size_t)(bi & 1) * S * rowbytes;
        const int j0 = bi * S;
#pragma unroll
        for (int r = 0; r < S; ++r) {
            if (j0 + r < cnt) {
                const uint32_t u = ids_s[j0 + r] & kIdMask;
                const unsigned char *row = rows + (size_t)u * rowbytes;
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    const int p = lane + 32 * c;
                    if (p < pieces) cp_async16(buf + r * rowbytes + p * 16, row + p * 16);
                }
                if constexpr (DT == 2) {
                    if (lane == r && scales) cp_async_small<4>(sbuf + (bi & 1) * S + r, scales + u);
                }
            }
        }
        cp_async_commit();
    };
    if (nb > 0) issue(0);
    for (int bi = 0; bi < nb; ++bi) {
        if (bi + 1 < nb) {
            __syncwarp();    // every lane has read the buffer scored two batches ago
            issue(bi + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();        // the other lanes' pieces of this batch have landed too
        const unsigned char *buf = cbuf + (size_t)(bi & 1) * S * rowbytes;
        const int j0 = bi * S;
        float sc[S];
#pragma unroll
        for (int r = 0; r < S; ++r) {
            sc[r] = 0.0f;
            const Chunk *rc = reinterpret_cast<const Chunk *>(buf + r * rowbytes);
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int ch = lane + 32 * c;
                if (ch < d4) {
                    RawChunk<DT> raw;
                    raw.v = rc[ch];
                    const float4 x = to_f4<DT>(raw);
                    sc[r] = fmaf(qr[c].x, x.x, sc[r]);
                    sc[r] = fmaf(qr[c].y, x.y, sc[r]);
                    sc[r] = fmaf(qr[c].z, x.z, sc[r]);
                    sc[r] = fmaf(qr[c].w, x.w, sc[r]);
                }
            }
        }
        const float mine = reduce_rows<S>(sc, lane);
        constexpr int RS = reduce_stride<S>();
        const int rr = lane / RS;
        if ((lane & (RS - 1)) == 0 && rr < S && j0 + rr < cnt) {
            if constexpr (DT == 2) {
                const float s8 = scales ? sbuf[(bi & 1) * S + rr] : 1.0f;
                out_s[j0 + rr] = -(s8 * mine);
            } else {
                out_s[j0 + rr] = -mine;
            }
        }
    }
    __syncwarp();
}

__device__ __forceinline__ uint32_t hash_slot(uint32_t u, int log2) {
    return (u * 2654435761u) >> (32 - log2);
}

// Shared-memory visited table. Returns 1 = newly inserted, 0 = already present,
// 2 = absent (lookup only), 3 = table full (cannot happen below half load).
__device__ __forceinline__ int smem_visit(uint32_t *tab, int log2, uint32_t u, bool insert) {
    const uint32_t mask = (1u << log2) - 1u;
    uint32_t h = hash_slot(u, log2);
    volatile uint32_t *vt = tab;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint32_t cur = vt[h];
        if (cur == u) return 0;
        if (cur == kNone) {
            if (!insert) return 2;
            const uint32_t old = atomicCAS(&tab[h], kNone, u);
            if (old == kNone) return 1;
            if (old == u) return 0;
        }
        h = (h + 1u) & mask;
    }
    return 3;
}

// Insert (cd_, ci_) at slot pos of a sorted pool of `size` entries with
// capacity L (pos < L, pos <= size): slots pos.. move up by one and the last
// falls off a full pool. Works on groups of 4 slots per lane (16-byte shared
// accesses, 128 slots per step) from the top down; the slot that crosses
// into the group above comes from the next lane by a shuffle (or, for the
// lowest group of a step, from shared memory below the step, not yet moved).
__device__ __forceinline__ void pool_insert_one(float *pd, uint32_t *pi, int size, int L, int pos,
                                                float cd_, uint32_t ci_, int lane) {
    const int last = min(size, L - 1);  // highest destination slot
    const int g_lo = pos >> 2, g_hi = last >> 2;
    float4 *pd4 = reinterpret_cast<float4 *>(pd);
    uint4 *pi4 = reinterpret_cast<uint4 *>(pi);
    for (int gb = g_hi; gb >= g_lo; gb -= 32) {
        const int g = gb - lane;
        const bool act = g >= g_lo;
        float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
        uint4 iv = make_uint4(0u, 0u, 0u, 0u);
        if (act) {
            dv = pd4[g];
            iv = pi4[g];
        }
        float pdv = __shfl_down_sync(kFull, dv.w, 1);
        uint32_t piv = __shfl_down_sync(kFull, iv.w, 1);
        if (act && (lane == 31 || g - 1 < g_lo) && g > 0) {
            pdv = pd[4 * g - 1];
            piv = pi[4 * g - 1];
        }
        if (act) {
            const int i0 = 4 * g;
            float4 nd = dv;
            uint4 ni = iv;
            // destination slot i takes the old slot i - 1 for pos < i <= last, the new entry at pos
#define ROAR_SLOT(J, PREVD, PREVI, DST_D, DST_I)                   \
    {                                                               \
        const int i = i0 + J;                                       \
        if (i == pos) { DST_D = cd_; DST_I = ci_; }                 \
        else if (i > pos && i <= last) { DST_D = PREVD; DST_I = PREVI; } \
    }
            ROAR_SLOT(0, pdv, piv, nd.x, ni.x)
            ROAR_SLOT(1, dv.x, iv.x, nd.y, ni.y)
            ROAR_SLOT(2, dv.y, iv.y, nd.z, ni.z)
            ROAR_SLOT(3, dv.z, iv.z, nd.w, ni.w)
#undef ROAR_SLOT
            pd4[g] = nd;
            pi4[g] = ni;
        }
        __syncwarp();
    }
}

// Global bitmap visited set: true if u was not yet set.
__device__ __forceinline__ bool bitmap_visit(uint32_t *bits, uint32_t u) {
    const uint32_t bit = 1u << (u & 31u);
    return (atomicOr(bits + (u >> 5), bit) & bit) == 0u;
}

// Number of entries of a sorted (d, id) array strictly before (dd, id).
__device__ __forceinline__ int lower_bound_entries(const float *dv, const uint32_t *iv, int size,
                                                   float dd, uint32_t id) {
    int lo = 0, hi = size;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (less_entry(dv[mid], iv[mid] & kIdMask, dd, id)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}


// Launch shape of a team of TW warps per query: CTAs of max(4, TW) warps,
// with the register budget of min_blocks_per_sm<DT, NCH>() 4-warp CTAs per SM.
template <int DT, int TW, int STG = 0, int NCH = 1>
struct TeamShape {
    static constexpr int kThreads = 32 * (TW > kWarpsPerBlock ? TW : kWarpsPerBlock);
    static constexpr int kTeams = kThreads / (32 * TW);
    static constexpr int kWarpBudget =
        (STG > 0 && DT == 0 ? ROAR_MIN_BLOCKS_STAGED : min_blocks_per_sm<DT, NCH>()) * kWarpsPerBlock;
    static constexpr int kMinBlocks = (kWarpBudget * 32) / kThreads > 0 ? (kWarpBudget * 32) / kThreads : 1;
};

// One query per team of TW warps. The leader warp (warp 0 of the team)
// selects, reads the adjacency row, updates the visited set and merges; all
// TW warps score the hop's new rows, each a strided share of whole dot
// products, so every distance is computed exactly as with one warp.
// RPL = adjacency ids per lane (rmax <= 32 * RPL), which also bounds the new
// candidates of one hop.
// STG > 0 (one warp per query): the hop's rows are gathered through shared
// memory, STG rows per buffer (score_rows_staged).
// BI (FP32, one warp): search on the bipartite graph G_bi. Expanding base
// node v walks its query nodes t in B(v) and processes the row N_out(t) of
// `adj` as one batch of candidates each (fetch, visited set, gather, merge)
// before the next selection; by the invariant above this is the same pool as
// merging all of v's two-hop neighbours at once. The visit cap is checked
// before each query node's row.
template <int DT, int NCH, int RPL, int TW, int STG, bool BI = false>
__global__ void __launch_bounds__(TeamShape<DT, TW, STG, NCH>::kThreads, TeamShape<DT, TW, STG, NCH>::kMinBlocks)
beam_search_kernel(const SearchArgs a) {
    static_assert(!BI || (DT == 0 && TW == 1 && STG == 0), "bipartite search: FP32, one warp, register gather");
    constexpr int kMaxRowPerLane = RPL;
    constexpr int kMaxCandPerLane = RPL;
    constexpr int TPB = TeamShape<DT, TW>::kTeams;
    constexpr int B = batch_rows<DT, NCH>();   // traversal rows per batch
    constexpr int B0 = rerank_rows<NCH>();     // FP32 re-rank rows per batch (BF16 / FP8 only)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int team = warp / TW;
    const int wt = warp - team * TW;
    const bool leader = wt == 0;
    const int lcap = a.lcap;
    const int hlog2 = a.hash_log2;           // 0: no shared table
    const int H = hlog2 ? (1 << hlog2) : 0;
    static_assert(STG == 0 || TW == 1, "staging is for one-warp kernels");
    constexpr int S = STG;  // staged gather rows per buffer (0: registers)
    const size_t stage = S ? stage_bytes(DT, S, a.d >> 2) : 0;
    unsigned char *tbase = smem_raw + (size_t)team * search_smem_per_team(lcap, hlog2, stage);
    unsigned char *stg = tbase + search_smem_per_team(lcap, hlog2, 0);
    float *pd = reinterpret_cast<float *>(tbase);
    uint32_t *pi = reinterpret_cast<uint32_t *>(pd + lcap);
    float *cd = reinterpret_cast<float *>(pi + lcap);
    uint32_t *ci = reinterpret_cast<uint32_t *>(cd + kCandCap);
    float *sd = reinterpret_cast<float *>(ci + kCandCap);
    uint32_t *si = reinterpret_cast<uint32_t *>(sd + kCandCap);
    uint32_t *htab = si + kCandCap;
    volatile int *ctl = reinterpret_cast<volatile int *>(htab + H);  // claim, count, size

    const int64_t slot = (int64_t)blockIdx.x * TPB + team;
    uint32_t *bits = a.vbits + slot * a.vbits_words;
    uint32_t *vlog = a.vlog + slot * (int64_t)a.vlog_cap;
    const int d = a.d, d4 = a.d >> 2;
    const int rmax = a.rmax;

    auto tsync = [&]() {
        if constexpr (TW == 1) {
            __syncwarp();
        } else {
            asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(TW * 32) : "memory");
        }
    };

    const bool serving = a.ring_pub != nullptr;
    const unsigned long long t_team0 = serving ? now_ns() : 0ull;   // idle floor (serving)
    for (;;) {
        if (leader && lane == 0) {
            if (!serving) {
                ctl[0] = (int)atomicAdd(a.work, 1u);
            } else {
                // Take the next ticket (a sequence number) with one atomicAdd,
                // or the ticket this team slot held when the last launch
                // exited, and wait (bounded) for its slot's publish mark. A
                // CAS loop on the head made every waiting team retry each
                // claim, and under load the claims were the serving limit.
                // Idle exit is one decision for the whole kernel: a team gives
                // up only when no team has been given a published ticket for
                // idle_polls microseconds (ring_clock[0], the global time of
                // the last one; a team's own start is the floor), and then
                // raises ring_clock[1] so that the others stop waiting too.
                // Its ticket is kept for the next launch; with exits per team,
                // a ticket kept by an exited team while others ran waited for
                // the whole kernel to time out.
                long long got = -1;
                unsigned long long t = *reinterpret_cast<volatile unsigned long long *>(a.ring_orphan + slot);
                if (t == ~0ull) t = atomicAdd(a.ring_head, 1ull);
                else a.ring_orphan[slot] = ~0ull;
                const unsigned long long idle_ns = 1000ull * a.idle_polls;
                volatile unsigned long long *clk = a.ring_clock;
                for (uint32_t spin = 0;; ++spin) {
                    if (*a.ring_stop) break;
                    if (__ldcg(a.ring_pub + (t % (unsigned long long)a.ring_cap)) == (uint32_t)(t + 1)) {
                        got = (long long)t;
                        clk[0] = now_ns();
                        break;
                    }
                    if ((spin & 15) == 0) {
                        if (clk[1]) break;
                        const unsigned long long now = now_ns(), last = clk[0];
                        if (now > (last > t_team0 ? last : t_team0) + idle_ns) {
                            clk[1] = 1ull;
                            break;
                        }
                    }
                    __nanosleep(1000);
                }
                if (got < 0) a.ring_orphan[slot] = t;
                __threadfence();  // the slot's data was written before its publish mark
                ctl[0] = (int)(got & 0xFFFFFFFF);
                ctl[3] = (int)(got >> 32);
            }
        }
        tsync();
        int64_t claim, qi;
        if (!serving) {
            claim = (int64_t)(unsigned)ctl[0];
            if (claim >= a.nq) break;
            qi = a.order ? (int64_t)a.order[claim] : claim;
        } else {
            claim = (int64_t)(((unsigned long long)(unsigned)ctl[3] << 32) | (unsigned)ctl[0]);
            if (claim < 0) break;
            qi = claim % a.ring_cap;
        }
        // A serving slot is one record (query, then k and L), rewritten when
        // the ring wraps: read it from L2.
        const float *rec = serving ? a.ring_rec + qi * (int64_t)a.ring_stride : nullptr;
        const int k = serving ? __ldcg(reinterpret_cast<const int *>(rec + d)) : (a.k_arr ? a.k_arr[qi] : a.k);
        const int L = serving ? __ldcg(reinterpret_cast<const int *>(rec + d) + 1) : (a.L_arr ? a.L_arr[qi] : a.L);
        const int64_t ooff = serving ? qi * (int64_t)a.ring_kmax : (a.out_off ? a.out_off[qi] : qi * (int64_t)k);
        if (L < 1 || L > lcap || k < 1 || k > L || (serving && k > a.ring_kmax)) {  // bad (k, L): report, skip
            if (leader && lane == 0) {
                if (a.visits) a.visits[qi] = 0;
                if (a.hops) a.hops[qi] = 0;
                if (a.qstatus) a.qstatus[qi] = ROAR_EINVAL;
                if (serving) {
                    __threadfence();
                    a.ring_done[qi] = (uint32_t)(claim + 1);
                }
            }
            continue;
        }

        float4 qr[NCH];
        const float4 *q4 = reinterpret_cast<const float4 *>(serving ? rec : a.q + qi * (int64_t)d);
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int ch = lane + 32 * c;
            qr[c] = ch < d4 ? (serving ? __ldcg(q4 + ch) : __ldg(q4 + ch)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // Leader-only search state.
        int64_t bi_j = 0, bi_end = 0;   // BI: query nodes of the base node being expanded
        int size = 1, cursor = 0, nlog = 0;
        uint32_t visits = 1, hops = 0, smem_count = 0;
        // Next-hop prediction (FP32 graph search): the adjacency row of the
        // second unexpanded entry at selection time is loaded during the hop
        // (a plain load, no side effect); it is the next node expanded unless
        // a new candidate overtakes it, and then its row is already in
        // registers. (Measured on GB300, 1M x 200: 3 % faster for FP32; the
        // BF16 / FP8 kernels, short of registers, were slower with it.)
        constexpr bool kPredict = !BI && DT == 0;
        uint32_t pred_v = kNone;
        uint32_t nbp[kMaxRowPerLane];
        bool spilled = (H == 0), bad = false, overflow = false;
        if (leader) {
            for (int i = lane; i < H; i += 32) htab[i] = kNone;
            __syncwarp();
            if (lane == 0) {
                if (spilled) {
                    bitmap_visit(bits, a.entry);
                    vlog[0] = a.entry;
                } else {
                    htab[hash_slot(a.entry, hlog2)] = a.entry;  // empty table: first probe is free
                }
                ci[0] = a.entry;
            }
            nlog = spilled ? 1 : 0;
            smem_count = spilled ? 0 : 1;
            __syncwarp();
            score_rows<DT, NCH, 1>(a.trav, a.scales, d, d4, qr, ci, 1, cd, lane);
            if (lane == 0) {
                pd[0] = cd[0];
                pi[0] = a.entry;
            }
            __syncwarp();
        }

        for (;;) {
            int cnt = 0;
            if (leader) {
                uint32_t v = 0;        // the adjacency row to read this round
                bool have_row = false;
                int sel2 = -1;         // the second unexpanded entry (same 32-entry block), or -1
                if (BI && bi_j < bi_end) {
                    // Next query node of the base node being expanded.
                    if (visits >= a.max_visits) {
                        overflow = true;
                        cnt = -1;
                    } else {
                        v = a.bi_q[bi_j++];
                        have_row = true;
                    }
                } else {
                    // Select: first unexpanded entry (all entries before `cursor` are expanded).
                    int sel = -1;
                    for (int b0 = cursor & ~31; b0 < size; b0 += 32) {
                        const int i = b0 + lane;
                        const bool open = i < size && !(pi[i] & kChecked);
                        const unsigned m = __ballot_sync(kFull, open);
                        if (m) {
                            sel = b0 + __ffs(m) - 1;
                            const unsigned m2 = m & (m - 1u);
                            if (m2) sel2 = b0 + __ffs(m2) - 1;
                            break;
                        }
                    }
                    if (sel >= 0 && visits >= a.max_visits) overflow = true;
                    if (sel < 0 || overflow) {
                        cnt = -1;
                    } else {
                        v = pi[sel] & kIdMask;
                        __syncwarp();
                        if (lane == 0) pi[sel] = v | kChecked;
                        ++hops;
                        if (a.trace && lane == 0 && hops <= (uint32_t)a.trace_cap) {
                            a.trace[qi * (int64_t)a.trace_cap + hops - 1] = v;
                            // the pool's L-th distance as this node is expanded (+inf while not full)
                            if (a.trace_bound)
                                a.trace_bound[qi * (int64_t)a.trace_cap + hops - 1] =
                                    size >= L ? pd[L - 1] : __int_as_float(0x7f800000);
                        }
                        cursor = sel + 1;
                        if constexpr (BI) {
                            bi_j = a.bi_off[v];
                            bi_end = a.bi_off[v + 1];
                            if (bi_j < bi_end) {
                                v = a.bi_q[bi_j++];
                                have_row = true;
                            }
                        } else {
                            have_row = true;
                        }
                    }
                }
                if (BI && have_row && (int64_t)v >= a.bi_nt) {   // a query id past the N_out table
                    bad = true;
                    have_row = false;
                }
                if (have_row) {
                    // Neighbour fetch + visited test-and-insert.
                    if (!spilled && (int)(smem_count + rmax) > (H >> 1)) spilled = true;
                    uint32_t nb[kMaxRowPerLane];
                    bool fresh[kMaxRowPerLane];
                    bool mybad = false;
                    if (kPredict && v == pred_v) {
#pragma unroll
                        for (int t = 0; t < kMaxRowPerLane; ++t) nb[t] = nbp[t];
                    } else {
#pragma unroll
                        for (int t = 0; t < kMaxRowPerLane; ++t) {
                            const int j = lane + 32 * t;
                            nb[t] = (j < rmax) ? __ldg(a.adj + (size_t)v * rmax + j) : kNone;
                        }
                    }
                    if constexpr (kPredict) {
                        pred_v = sel2 >= 0 ? (pi[sel2] & kIdMask) : kNone;
                        if (pred_v != kNone) {
#pragma unroll
                            for (int t = 0; t < kMaxRowPerLane; ++t) {
                                const int j = lane + 32 * t;
                                nbp[t] = (j < rmax) ? __ldg(a.adj + (size_t)pred_v * rmax + j) : kNone;
                            }
                        }
                    }
#pragma unroll
                    for (int t = 0; t < kMaxRowPerLane; ++t) {
                        fresh[t] = false;
                        const uint32_t u = nb[t];
                        if (u == kNone) continue;
                        if ((int64_t)u >= a.n) {
                            mybad = true;
                            continue;
                        }
                        if (!spilled) {
                            fresh[t] = smem_visit(htab, hlog2, u, true) == 1;
                        } else if (H == 0 || smem_visit(htab, hlog2, u, false) == 2) {
                            fresh[t] = bitmap_visit(bits, u);
                        }
                    }
                    if (__any_sync(kFull, mybad)) bad = true;
#pragma unroll
                    for (int t = 0; t < kMaxRowPerLane; ++t) {
                        const unsigned m = __ballot_sync(kFull, fresh[t]);
                        if (fresh[t]) ci[cnt + __popc(m & ((1u << lane) - 1u))] = nb[t];
                        cnt += __popc(m);
                    }
                    __syncwarp();
                    if (ROAR_PREFETCH_ROWS) prefetch_rows_l2(a.trav, (uint32_t)d * (4u >> DT), ci, cnt, lane);
                    if (spilled) {  // every fresh id this hop went to the bitmap: log it
                        for (int j = lane; j < cnt; j += 32) vlog[nlog + j] = ci[j];
                        nlog += cnt;
                    } else {
                        smem_count += cnt;
                    }
                    visits += cnt;
                }
                if (lane == 0) {
                    ctl[1] = cnt;
                    ctl[2] = size;
                }
            }
            tsync();
            cnt = ctl[1];
            if (cnt < 0) break;
            if (cnt == 0) continue;

            // Gather + score: warp wt takes row groups wt, wt + TW, ...
            if constexpr (S > 0) {
                score_rows_staged<DT, NCH, S>(a.trav, a.scales, d4, qr, ci, cnt, cd, lane, stg);
            } else {
                score_rows<DT, NCH, B>(a.trav, a.scales, d, d4, qr, ci, cnt, cd, lane, wt * B, TW * B);
            }
            tsync();
            if (!leader) continue;

            // Drop candidates that cannot enter a full pool.
            if (size == L) {
                const float wd = pd[L - 1];
                const uint32_t wi = pi[L - 1] & kIdMask;
                float kd[kMaxCandPerLane];
                uint32_t kid[kMaxCandPerLane];
                bool keep[kMaxCandPerLane];
#pragma unroll
                for (int t = 0; t < kMaxCandPerLane; ++t) {
                    const int j = lane + 32 * t;
                    keep[t] = false;
                    if (j < cnt) {
                        kd[t] = cd[j];
                        kid[t] = ci[j];
                        keep[t] = less_entry(kd[t], kid[t], wd, wi);
                    }
                }
                __syncwarp();
                int c2 = 0;
#pragma unroll
                for (int t = 0; t < kMaxCandPerLane; ++t) {
                    const unsigned m = __ballot_sync(kFull, keep[t]);
                    if (keep[t]) {
                        const int p = c2 + __popc(m & ((1u << lane) - 1u));
                        cd[p] = kd[t];
                        ci[p] = kid[t];
                    }
                    c2 += __popc(m);
                }
                cnt = c2;
                __syncwarp();
                if (cnt == 0) continue;
            }
            // Sort the candidates (ids are distinct, so ranks are a permutation).
#pragma unroll
            for (int t = 0; t < kMaxCandPerLane; ++t) {
                const int j = lane + 32 * t;
                if (j < cnt) {
                    const float dj = cd[j];
                    const uint32_t ij = ci[j];
                    int r = 0;
                    for (int x = 0; x < cnt; ++x) r += less_entry(cd[x], ci[x], dj, ij) ? 1 : 0;
                    sd[r] = dj;
                    si[r] = ij;
                }
            }
            __syncwarp();
            // Final slot of sorted candidate r: (#pool entries before it) + r.
            int cpos[kMaxCandPerLane];
#pragma unroll
            for (int t = 0; t < kMaxCandPerLane; ++t) {
                const int r = lane + 32 * t;
                cpos[t] = r < cnt ? lower_bound_entries(pd, pi, size, sd[r], si[r]) + r : 0x7FFFFFFF;
            }
            const int pmin = __shfl_sync(kFull, cpos[0], 0);
            if (cnt <= 4) {
                // Few candidates (the usual case once the pool is full): insert
                // them one at a time in increasing slot order. (A single
                // destination-driven pass for all of them measured 1-2 % slower
                // on GB300: its scalar shared-memory reads conflict on banks.)
                int sz = size;
                for (int r = 0; r < cnt; ++r) {
                    const int pos = __shfl_sync(kFull, cpos[0], r);
                    if (pos >= L) break;
                    pool_insert_one(pd, pi, sz, L, pos, sd[r], si[r], lane);
                    sz = min(L, sz + 1);
                }
                size = sz;
                cursor = min(cursor, pmin);
                __syncwarp();
                continue;
            }
            // Many candidates: move the pool tail [pmin, size) up in place, 32
            // entries at a time from the end: new slots are increasing and never
            // below the old ones, so no write lands on an entry not yet read.
            for (int hi = size; hi > pmin; hi -= 32) {
                const int i = hi - 32 + lane;
                const bool act = i >= pmin;
                float di = 0.f;
                uint32_t ii = 0;
                int np = 0;
                if (act) {
                    di = pd[i];
                    ii = pi[i];
                    np = i + lower_bound_entries(sd, si, cnt, di, ii & kIdMask);
                }
                __syncwarp();
                if (act && np < L) {
                    pd[np] = di;
                    pi[np] = ii;
                }
                __syncwarp();
            }
#pragma unroll
            for (int t = 0; t < kMaxCandPerLane; ++t) {
                const int r = lane + 32 * t;
                if (r < cnt && cpos[t] < L) {
                    pd[cpos[t]] = sd[r];
                    pi[cpos[t]] = si[r];
                }
            }
            size = min(L, size + cnt);
            cursor = min(cursor, pmin);
            __syncwarp();
        }

        // Output (re-ranked in FP32, in place, for the reduced-precision forms).
        // Deleted rows (tombstones) took part in routing and are skipped here.
        const int fsize = ctl[2];
        auto deleted = [&](uint32_t u) -> bool { return (__ldcg(a.tomb + (u >> 5)) >> (u & 31)) & 1u; };
        if constexpr (DT != 0) {
            // The pool's FP32 rows are asked of L2 a few batches ahead (all at
            // once would be evicted before use for long pools).
            score_rows<0, NCH, B0>(a.base32, nullptr, d, d4, qr, pi, fsize, pd, lane, wt * B0, TW * B0,
                                   (16 + B0 - 1) / B0);
            tsync();
            if (leader) {
                int alive = fsize;
                if (a.tomb) {  // a deleted entry ranks after every live one and is not written
                    alive = 0;
                    for (int b0 = 0; b0 < fsize; b0 += 32) {
                        const int i = b0 + lane;
                        const bool dead = i < fsize && deleted(pi[i] & kIdMask);
                        if (dead) pd[i] = __int_as_float(0x7f800000);
                        alive += __popc(__ballot_sync(kFull, i < fsize && !dead));
                    }
                    __syncwarp();
                }
                for (int i = lane; i < fsize; i += 32) {
                    const float di = pd[i];
                    const uint32_t ii = pi[i] & kIdMask;
                    if (a.tomb && deleted(ii)) continue;
                    int r = 0;
                    for (int x = 0; x < fsize && r < k; ++x)
                        r += less_entry(pd[x], pi[x] & kIdMask, di, ii) ? 1 : 0;
                    if (r < k) {
                        a.ids[ooff + r] = ii;
                        a.dist[ooff + r] = di;
                    }
                }
                for (int r = alive + lane; r < k; r += 32) {
                    a.ids[ooff + r] = kNone;
                    a.dist[ooff + r] = __int_as_float(0x7f800000);
                }
            }
        } else if (leader) {
            if (!a.tomb) {
                for (int r = lane; r < k; r += 32) {
                    const bool have = r < fsize;
                    a.ids[ooff + r] = have ? (pi[r] & kIdMask) : kNone;
                    a.dist[ooff + r] = have ? pd[r] : __int_as_float(0x7f800000);
                }
            } else {  // the first k live pool entries, in pool order
                int r = 0;
                for (int b0 = 0; b0 < fsize && r < k; b0 += 32) {
                    const int i = b0 + lane;
                    const uint32_t u = i < fsize ? (pi[i] & kIdMask) : 0u;
                    const bool live = i < fsize && !deleted(u);
                    const unsigned m = __ballot_sync(kFull, live);
                    const int p = r + __popc(m & ((1u << lane) - 1u));
                    if (live && p < k) {
                        a.ids[ooff + p] = u;
                        a.dist[ooff + p] = pd[i];
                    }
                    r += __popc(m);
                }
                for (int p = min(r, k) + lane; p < k; p += 32) {
                    a.ids[ooff + p] = kNone;
                    a.dist[ooff + p] = __int_as_float(0x7f800000);
                }
            }
        }
        if (leader) {
            __syncwarp();  // orders every lane's result writes before lane 0's fence below
            if (lane == 0) {
                if (a.visits) a.visits[qi] = visits;
                if (a.hops) a.hops[qi] = hops;
                if (a.qstatus) a.qstatus[qi] = overflow ? ROAR_EOVERFLOW : (bad ? ROAR_EINVAL : ROAR_OK);
                if (serving) {  // the results (cumulative over the warp) before the done mark
                    __threadfence();
                    a.ring_done[qi] = (uint32_t)(claim + 1);
                }
            }
            // Return the bitmap to all-zero: clear every word this query set.
            // The bitmap belongs to this warp, so plain stores do (the
            // __syncwarp orders them before the next query's atomics); the
            // log is read 4 entries per lane at a time, so the loads overlap.
            for (int i0 = 0; i0 < nlog; i0 += 128) {
                uint32_t w[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int i = i0 + 32 * j + lane;
                    w[j] = i < nlog ? __ldcg(vlog + i) : kNone;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (w[j] != kNone) bits[w[j] >> 5] = 0u;
            }
            __syncwarp();
        }
    }
}

}  // namespace

// Kernel for (row chunks per lane, adjacency ids per lane, warps per team,
// staged gather: one-warp kernels only).
template <int DT>
const void *kernel_table(int nch, int rpl, int tw, bool staged) {
#define ROAR_K(N, R, T) \
    if (nch == N && rpl == R && tw == T && !staged) return (const void *)beam_search_kernel<DT, N, R, T, 0>;
#define ROAR_KS(N, R)                                                                              \
    if constexpr (stage_rows(DT, N) > 0) {                                                         \
        if (nch == N && rpl == R && tw == 1 && staged)                                             \
            return (const void *)beam_search_kernel<DT, N, R, 1, stage_rows(DT, N)>;               \
    }
#define ROAR_KT(N, R) ROAR_K(N, R, 1) ROAR_K(N, R, 2) ROAR_K(N, R, 4) ROAR_K(N, R, 8) ROAR_KS(N, R)
#define ROAR_KN(N) ROAR_KT(N, 2) ROAR_KT(N, 4)
    ROAR_KN(1) ROAR_KN(2) ROAR_KN(4) ROAR_KN(8)
#undef ROAR_KN
#undef ROAR_KT
#undef ROAR_KS
#undef ROAR_K
    return nullptr;
}

// Bipartite-graph kernels (FP32, one warp), instantiated by the FP32 unit.
template <int DT>
const void *kernel_table_bi_t(int nch, int rpl) {
    static_assert(DT == 0, "bipartite search is FP32");
#define ROAR_KB(N, R) \
    if (nch == N && rpl == R) return (const void *)beam_search_kernel<DT, N, R, 1, 0, true>;
    ROAR_KB(1, 2) ROAR_KB(1, 4) ROAR_KB(2, 2) ROAR_KB(2, 4) ROAR_KB(4, 2) ROAR_KB(4, 4) ROAR_KB(8, 2) ROAR_KB(8, 4)
#undef ROAR_KB
    return nullptr;
}

}  // namespace roar
