// Batched beam search over a RoarGraph index (Sec. 4.3), one warp per query.
//
// Per warp, in shared memory: the size-L candidate pool sorted by
// (distance, id) with an "expanded" bit in each id, a scratch copy used by
// the merge, the new candidates of the current hop, and an exact visited set
// (open addressing, linear probing). When a query visits more nodes than the
// shared table holds at half load, further inserts go to an exact per-warp
// table in global memory whose entries carry a per-query tag, so it never
// needs clearing.
//
// Each hop: pick the first unexpanded pool entry, read its adjacency row
// (coalesced, one id per lane), filter and insert the neighbours into the
// visited set, gather the new rows and score them with a warp-cooperative dot
// product in one fixed order, then merge the scored candidates into the pool.
// The fixed order (element i to lane (i >> 2) & 31, fmaf per lane in
// increasing i, then s += shfl_xor(s, o) for o = 16, 8, 4, 2, 1) is exactly
// what a float4 load per lane produces, and makes every distance, and hence
// the whole trajectory, independent of the batch and of the launch shape.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "roar_internal.cuh"

namespace roar {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ bool less_entry(float da, uint32_t ia, float db, uint32_t ib) {
    return da < db || (da == db && ia < ib);
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

// Raw row chunk (4 elements) of row u, chunk ch, in the traversal format.
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

// Distances for cnt rows whose ids are in ids_s (shared); writes -<q, x> (times
// the row scale for FP8) to out_s. Rows are processed B at a time so each lane
// has B * NCH independent loads in flight.
template <int DT, int NCH, int B>
__device__ __forceinline__ void score_rows(const void *base, const float *scales, int d, int d4,
                                           const float4 (&qr)[NCH], const uint32_t *ids_s, int cnt,
                                           float *out_s, int lane) {
    for (int j0 = 0; j0 < cnt; j0 += B) {
        RawChunk<DT> raw[B][NCH];
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
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
            for (int b = 0; b < B; ++b) s[b] = s[b] + __shfl_xor_sync(kFull, s[b], o);
        }
        if (lane < B && j0 + lane < cnt) {
            float mine = s[0];
#pragma unroll
            for (int b = 1; b < B; ++b)
                if (lane == b) mine = s[b];
            if constexpr (DT == 2) {
                const float sc = scales ? __ldg(scales + (ids_s[j0 + lane] & kIdMask)) : 1.0f;
                out_s[j0 + lane] = -(sc * mine);
            } else {
                out_s[j0 + lane] = -mine;
            }
        }
    }
    __syncwarp();
}

__device__ __forceinline__ uint32_t hash_slot(uint32_t u, int log2) {
    return (u * 2654435761u) >> (32 - log2);
}

// Shared-memory visited set. Returns 1 = newly inserted, 0 = already present,
// 2 = absent (lookup only), 3 = table full (cannot happen below half load).
__device__ __forceinline__ int smem_visit(uint32_t *tab, int log2, uint32_t u, bool insert) {
    const uint32_t mask = (1u << log2) - 1u;
    uint32_t h = hash_slot(u, log2);
    volatile uint32_t *vt = tab;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        uint32_t cur = vt[h];
        if (cur == u) return 0;
        if (cur == kNone) {
            if (!insert) return 2;
            uint32_t old = atomicCAS(&tab[h], kNone, u);
            if (old == kNone) return 1;
            if (old == u) return 0;
        }
        h = (h + 1u) & mask;
    }
    return 3;
}

// Global overflow visited set; entry = (tag << 32) | id, live iff tag == epoch.
__device__ __forceinline__ int global_visit(unsigned long long *tab, int log2, uint32_t epoch,
                                            uint32_t u) {
    const uint32_t mask = (1u << log2) - 1u;
    uint32_t h = hash_slot(u, log2);
    const unsigned long long want = ((unsigned long long)epoch << 32) | u;
    volatile unsigned long long *vt = tab;
    for (uint32_t probe = 0; probe <= mask;) {
        unsigned long long cur = vt[h];
        if ((uint32_t)(cur >> 32) == epoch) {
            if ((uint32_t)cur == u) return 0;
            h = (h + 1u) & mask;
            ++probe;
            continue;
        }
        unsigned long long old = atomicCAS(&tab[h], cur, want);
        if (old == cur) return 1;
        // the slot changed under us: look at it again
    }
    return 3;
}

// Number of pool entries strictly before (dd, id) in the total order.
__device__ __forceinline__ int pool_lower_bound(const float *pd, const uint32_t *pi, int size,
                                                float dd, uint32_t id) {
    int lo = 0, hi = size;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (less_entry(pd[mid], pi[mid] & kIdMask, dd, id)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Rows gathered per batch: about 8 16-byte loads in flight per lane.
template <int NCH>
__host__ __device__ constexpr int batch_rows() {
    return NCH >= 8 ? 1 : 8 / NCH;
}

template <int DT, int NCH>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 4)
beam_search_kernel(const SearchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int lcap = a.lcap;
    unsigned char *wbase = smem_raw + (size_t)wib * search_smem_per_warp(lcap, a.hash_log2);
    float *pd = reinterpret_cast<float *>(wbase);
    uint32_t *pi = reinterpret_cast<uint32_t *>(pd + lcap);
    float *td = reinterpret_cast<float *>(pi + lcap);
    uint32_t *ti = reinterpret_cast<uint32_t *>(td + lcap);
    float *cd = reinterpret_cast<float *>(ti + lcap);
    uint32_t *ci = reinterpret_cast<uint32_t *>(cd + kCandCap);
    float *sd = reinterpret_cast<float *>(ci + kCandCap);
    uint32_t *si = reinterpret_cast<uint32_t *>(sd + kCandCap);
    uint32_t *htab = si + kCandCap;
    const int hlog2 = a.hash_log2;
    const int H = 1 << hlog2;

    const int slot = blockIdx.x * kWarpsPerBlock + wib;
    unsigned long long *gtab = a.spill + ((size_t)slot << a.spill_log2);
    const int S = 1 << a.spill_log2;
    uint32_t epoch = a.slot_epoch[slot];
    const int d = a.d, d4 = a.d >> 2;
    const int rmax = a.rmax;

    for (;;) {
        unsigned int qclaim = 0;
        if (lane == 0) qclaim = atomicAdd(a.work, 1u);
        qclaim = __shfl_sync(kFull, qclaim, 0);
        const int64_t qi = (int64_t)qclaim;
        if (qi >= a.nq) break;
        const int k = a.k_arr ? a.k_arr[qi] : a.k;
        const int L = a.L_arr ? a.L_arr[qi] : a.L;
        const int64_t ooff = a.out_off ? a.out_off[qi] : qi * (int64_t)k;

        if (++epoch == 0u) {  // tag wrapped: old entries could alias, clear once
            for (int i = lane; i < S; i += 32) gtab[i] = 0ull;
            epoch = 1u;
            __threadfence_block();
        }
        for (int i = lane; i < H; i += 32) htab[i] = kNone;
        __syncwarp();

        float4 qr[NCH];
        const float4 *q4 = reinterpret_cast<const float4 *>(a.q + qi * (int64_t)d);
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int ch = lane + 32 * c;
            qr[c] = ch < d4 ? __ldg(q4 + ch) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (lane == 0) {
            htab[hash_slot(a.entry, hlog2)] = a.entry;  // empty table: first probe is free
            ci[0] = a.entry;
        }
        __syncwarp();
        score_rows<DT, NCH, 1>(a.trav, a.scales, d, d4, qr, ci, 1, cd, lane);
        if (lane == 0) {
            pd[0] = cd[0];
            pi[0] = a.entry;
        }
        __syncwarp();

        int size = 1, cursor = 0;
        uint32_t visits = 1, hops = 0, smem_count = 1;
        bool spilled = false, bad = false, overflow = false;

        for (;;) {
            // Select: first unexpanded entry (all entries before `cursor` are expanded).
            int sel = -1;
            for (int b0 = cursor & ~31; b0 < size; b0 += 32) {
                const int i = b0 + lane;
                const bool open = i < size && !(pi[i] & kChecked);
                const unsigned m = __ballot_sync(kFull, open);
                if (m) {
                    sel = b0 + __ffs(m) - 1;
                    break;
                }
            }
            if (sel < 0) break;
            if (visits >= a.max_visits) {
                overflow = true;
                break;
            }
            const uint32_t v = pi[sel] & kIdMask;
            __syncwarp();
            if (lane == 0) pi[sel] = v | kChecked;
            ++hops;
            cursor = sel + 1;

            // Neighbour fetch + visited filter.
            if (!spilled && (int)(smem_count + rmax) > (H >> 1)) spilled = true;
            uint32_t nb[kMaxRowPerLane];
            bool fresh[kMaxRowPerLane];
            bool mybad = false;
#pragma unroll
            for (int t = 0; t < kMaxRowPerLane; ++t) {
                const int j = lane + 32 * t;
                nb[t] = (j < rmax) ? __ldg(a.adj + (size_t)v * rmax + j) : kNone;
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
                } else {
                    const int r = smem_visit(htab, hlog2, u, false);
                    if (r == 2) fresh[t] = global_visit(gtab, a.spill_log2, epoch, u) == 1;
                }
            }
            if (__any_sync(kFull, mybad)) bad = true;
            int cnt = 0;
#pragma unroll
            for (int t = 0; t < kMaxRowPerLane; ++t) {
                const unsigned m = __ballot_sync(kFull, fresh[t]);
                if (fresh[t]) ci[cnt + __popc(m & ((1u << lane) - 1u))] = nb[t];
                cnt += __popc(m);
            }
            visits += cnt;
            if (!spilled) smem_count += cnt;
            __syncwarp();
            if (cnt == 0) continue;

            // Gather + score.
            score_rows<DT, NCH, batch_rows<NCH>()>(a.trav, a.scales, d, d4, qr, ci, cnt, cd, lane);

            // Merge: drop candidates that cannot enter a full pool.
            if (size == L) {
                const float wd = pd[L - 1];
                const uint32_t wi = pi[L - 1] & kIdMask;
                float kd[kMaxRowPerLane];
                uint32_t kid[kMaxRowPerLane];
                bool keep[kMaxRowPerLane];
#pragma unroll
                for (int t = 0; t < kMaxRowPerLane; ++t) {
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
                for (int t = 0; t < kMaxRowPerLane; ++t) {
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
            // Rank candidates among themselves (ids are distinct).
#pragma unroll
            for (int t = 0; t < kMaxRowPerLane; ++t) {
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
            // Entries before the first candidate's slot stay where they are.
            const int pmin = pool_lower_bound(pd, pi, size, sd[0], si[0]);
            for (int i = pmin + lane; i < size; i += 32) {
                td[i] = pd[i];
                ti[i] = pi[i];
            }
            __syncwarp();
            for (int i = pmin + lane; i < size; i += 32) {
                const float di = td[i];
                const uint32_t ii = ti[i];
                int lo = 0, hi = cnt;  // candidates before this pool entry
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (less_entry(sd[mid], si[mid], di, ii & kIdMask)) lo = mid + 1;
                    else hi = mid;
                }
                const int np = i + lo;
                if (np < L) {
                    pd[np] = di;
                    pi[np] = ii;
                }
            }
            // Candidate r lands at (#pool entries before it) + r. Pool entries
            // before pmin are unchanged in pd/pi; those from pmin are in td/ti.
            for (int r = lane; r < cnt; r += 32) {
                const float dr = sd[r];
                const uint32_t ir = si[r];
                int lo = pmin, hi = size;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (less_entry(td[mid], ti[mid] & kIdMask, dr, ir)) lo = mid + 1;
                    else hi = mid;
                }
                const int np = lo + r;
                if (np < L) {
                    pd[np] = dr;
                    pi[np] = ir;
                }
            }
            size = min(L, size + cnt);
            cursor = min(cursor, pmin);
            __syncwarp();
        }

        // Output (re-ranked in FP32 for the reduced-precision forms).
        if constexpr (DT != 0) {
            for (int i = lane; i < size; i += 32) ti[i] = pi[i] & kIdMask;
            __syncwarp();
            score_rows<0, NCH, batch_rows<NCH>()>(a.base32, nullptr, d, d4, qr, ti, size, td, lane);
            for (int i = lane; i < size; i += 32) {
                const float di = td[i];
                const uint32_t ii = ti[i];
                int r = 0;
                for (int x = 0; x < size && r < k; ++x) r += less_entry(td[x], ti[x], di, ii) ? 1 : 0;
                if (r < k) {
                    a.ids[ooff + r] = ii;
                    a.dist[ooff + r] = di;
                }
            }
            for (int r = size + lane; r < k; r += 32) {
                a.ids[ooff + r] = kNone;
                a.dist[ooff + r] = __int_as_float(0x7f800000);
            }
        } else {
            for (int r = lane; r < k; r += 32) {
                const bool have = r < size;
                a.ids[ooff + r] = have ? (pi[r] & kIdMask) : kNone;
                a.dist[ooff + r] = have ? pd[r] : __int_as_float(0x7f800000);
            }
        }
        if (lane == 0) {
            if (a.visits) a.visits[qi] = visits;
            if (a.hops) a.hops[qi] = hops;
            if (a.qstatus) a.qstatus[qi] = overflow ? ROAR_EOVERFLOW : (bad ? ROAR_EINVAL : ROAR_OK);
        }
        __syncwarp();
    }
    if (lane == 0) a.slot_epoch[slot] = epoch;
}

template <int DT>
const void *kernel_for(int nch) {
    switch (nch) {
        case 1: return (const void *)beam_search_kernel<DT, 1>;
        case 2: return (const void *)beam_search_kernel<DT, 2>;
        case 3: return (const void *)beam_search_kernel<DT, 3>;
        case 4: return (const void *)beam_search_kernel<DT, 4>;
        case 5: return (const void *)beam_search_kernel<DT, 5>;
        case 6: return (const void *)beam_search_kernel<DT, 6>;
        case 7: return (const void *)beam_search_kernel<DT, 7>;
        case 8: return (const void *)beam_search_kernel<DT, 8>;
        default: return nullptr;
    }
}

const void *search_kernel(int dtype, int d) {
    const int nch = ((d >> 2) + 31) / 32;
    switch (dtype) {
        case 0: return kernel_for<0>(nch);
        case 1: return kernel_for<1>(nch);
        case 2: return kernel_for<2>(nch);
        default: return nullptr;
    }
}

}  // namespace

int hash_log2_for(int L) {
    const int lcap = (L + 31) / 32 * 32;
    const size_t budget = 227 * 1024;  // opt-in shared memory per CTA
    int lg = 10;
    while ((1 << lg) < 32 * L && lg < 14) ++lg;
    // Prefer 4 resident CTAs per SM (the register-bound maximum), then at least one.
    while (lg > 9 && search_smem_per_warp(lcap, lg) * kWarpsPerBlock * 4 > budget) --lg;
    while (lg > 5 && search_smem_per_warp(lcap, lg) * kWarpsPerBlock > budget) --lg;
    return lg;
}

int search_blocks_per_sm(int dtype, int d, int lcap, int hash_log2) {
    const void *fn = search_kernel(dtype, d);
    if (!fn) return 0;
    const size_t smem = search_smem_per_warp(lcap, hash_log2) * kWarpsPerBlock;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, kWarpsPerBlock * 32, smem) !=
        cudaSuccess)
        return 0;
    return blocks < kMaxWarpsPerSm / kWarpsPerBlock ? blocks : kMaxWarpsPerSm / kWarpsPerBlock;
}

cudaError_t launch_search(const SearchArgs &a, int blocks, cudaStream_t s) {
    const void *fn = search_kernel(a.dtype, a.d);
    if (!fn || blocks <= 0) return cudaErrorInvalidValue;
    const size_t smem = search_smem_per_warp(a.lcap, a.hash_log2) * kWarpsPerBlock;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(a.work, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<SearchArgs *>(&a)};
    return cudaLaunchKernel(fn, dim3(blocks), dim3(kWarpsPerBlock * 32), args, smem, s);
}

}  // namespace roar
