// AcquireNeighbors (Alg. 3, Sec. 4.2.3) for many nodes at once on the GPU: the
// pruning step of index construction (projection and connectivity
// enhancement keep, for node x, the candidates c that are closer to x than to
// every neighbour already kept).
//
// One warp per node x:
//   1. delta(x, c) = -dot(x, c) for every candidate, in the search's fixed FP32
//      order (score_rows: element i on lane (i >> 2) & 31, fmaf, xor
//      butterfly), padding ids (0xFFFFFFFF) dropped;
//   2. the candidates sorted by (delta, id) in shared memory (bitonic sort);
//   3. Alg. 3 in that order: skip x itself and ids already kept; keep the
//      first; keep any later c with delta(x, c) < delta(c, r) for every kept r,
//      where delta(c, r) for all kept r comes from one batched score_rows call
//      with c as the query; stop at M; with fill, top up to M from the
//      remaining candidates in order.
// Every decision is taken in FP32 with those exact sums, so the result is
// defined without reference to any particular sort or launch shape.
#include <algorithm>

#include "roar_search_kernel.cuh"

namespace roar {
roar_status cuda_fail(cudaError_t e, const char *what);
void set_error(const char *msg);
bool aligned(const void *p, size_t a);
}  // namespace roar

namespace roar {
namespace {

constexpr int kAcqWarps = 4;        // warps (nodes in flight) per CTA
constexpr int kAcqMaxCand = 1024;   // candidates per node (sort capacity)
constexpr int kAcqMaxM = 64;        // kept neighbours per node

struct AcqSmem {                    // per warp
    float cd[kAcqMaxCand];
    uint32_t ci[kAcqMaxCand];
    float rd[kAcqMaxM];
    uint32_t res[kAcqMaxM];
};

__device__ __forceinline__ bool acq_less(float da, uint32_t ia, float db, uint32_t ib) {
    return da < db || (da == db && ia < ib);
}

template <int NCH>
__device__ __forceinline__ void load_query(const float *X, uint32_t u, int d4, float4 (&qr)[NCH], int lane) {
    const float4 *r = reinterpret_cast<const float4 *>(X) + (size_t)u * d4;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        const int ch = lane + 32 * c;
        qr[c] = ch < d4 ? __ldg(r + ch) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <int NCH>
__global__ void __launch_bounds__(32 * kAcqWarps)
acquire_kernel(const float *__restrict__ X, int64_t n, int d, const uint32_t *__restrict__ xs, int64_t nx,
               const uint32_t *__restrict__ cand, int cstride, const int32_t *__restrict__ ncand, int M,
               int fill, uint32_t *__restrict__ out, int32_t *__restrict__ out_cnt,
               uint32_t *__restrict__ sorted_out) {
    constexpr int B = batch_rows<0, NCH>();
    __shared__ AcqSmem sm[kAcqWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    AcqSmem &S = sm[w];
    const int d4 = d >> 2;
    for (int64_t i = (int64_t)blockIdx.x * kAcqWarps + w; i < nx; i += (int64_t)gridDim.x * kAcqWarps) {
        const uint32_t x = xs[i];
        const int nc = min(max(ncand[i], 0), cstride);
        const uint32_t *ci_g = cand + (size_t)i * cstride;
        // 0. validate and compact the candidate ids (padding dropped).
        bool bad = (int64_t)x >= n;
        int nv = 0;
        for (int b0 = 0; b0 < nc; b0 += 32) {
            const int j = b0 + lane;
            const uint32_t u = j < nc ? ci_g[j] : kNone;
            if (u != kNone && (int64_t)u >= n) bad = true;
            const bool ok = u != kNone && (int64_t)u < n;
            const unsigned m = __ballot_sync(kFull, ok);
            if (ok) S.ci[nv + __popc(m & ((1u << lane) - 1u))] = u;
            nv += __popc(m);
        }
        if (__any_sync(kFull, bad)) {
            for (int j = lane; j < M; j += 32) out[(size_t)i * M + j] = kNone;
            if (sorted_out)
                for (int j = lane; j < cstride; j += 32) sorted_out[(size_t)i * cstride + j] = kNone;
            if (lane == 0) out_cnt[i] = -1;
            __syncwarp();
            continue;
        }
        __syncwarp();
        // 1. delta(x, c) for every candidate.
        float4 qr[NCH];
        load_query<NCH>(X, x, d4, qr, lane);
        score_rows<0, NCH, B>(X, nullptr, d, d4, qr, S.ci, nv, S.cd, lane);
        // 2. bitonic sort of (cd, ci) over the next power of two, padded with (+inf, kNone).
        int P = 1;
        while (P < nv) P <<= 1;
        for (int j = nv + lane; j < P; j += 32) {
            S.cd[j] = __int_as_float(0x7f800000);
            S.ci[j] = kNone;
        }
        __syncwarp();
        for (int k = 2; k <= P; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = lane; t < P; t += 32) {
                    const int o = t ^ j;
                    if (o > t) {
                        const float da = S.cd[t], db = S.cd[o];
                        const uint32_t ia = S.ci[t], ib = S.ci[o];
                        const bool up = (t & k) == 0;
                        if (up ? acq_less(db, ib, da, ia) : acq_less(da, ia, db, ib)) {
                            S.cd[t] = db;
                            S.cd[o] = da;
                            S.ci[t] = ib;
                            S.ci[o] = ia;
                        }
                    }
                }
                __syncwarp();
            }
        }
        // 3. Alg. 3 over the sorted candidates.
        int nr = 0;
        for (int t = 0; t < nv && nr < M; ++t) {
            const uint32_t c = S.ci[t];
            if (c == x) continue;
            const bool dupl = (lane < nr && S.res[lane] == c) || (lane + 32 < nr && S.res[lane + 32] == c);
            if (__any_sync(kFull, dupl)) continue;
            if (nr > 0) {
                float4 qc[NCH];
                load_query<NCH>(X, c, d4, qc, lane);
                score_rows<0, NCH, B>(X, nullptr, d, d4, qc, S.res, nr, S.rd, lane);
                const float dc = S.cd[t];
                const bool viol = (lane < nr && !(dc < S.rd[lane])) || (lane + 32 < nr && !(dc < S.rd[lane + 32]));
                if (__any_sync(kFull, viol)) continue;
            }
            if (lane == 0) S.res[nr] = c;
            ++nr;
            __syncwarp();
        }
        if (fill) {
            for (int t = 0; t < nv && nr < M; ++t) {
                const uint32_t c = S.ci[t];
                if (c == x) continue;
                const bool dupl = (lane < nr && S.res[lane] == c) || (lane + 32 < nr && S.res[lane + 32] == c);
                if (__any_sync(kFull, dupl)) continue;
                if (lane == 0) S.res[nr] = c;
                ++nr;
                __syncwarp();
            }
        }
        // 4. outputs.
        for (int j = lane; j < M; j += 32) out[(size_t)i * M + j] = j < nr ? S.res[j] : kNone;
        if (sorted_out)
            for (int j = lane; j < cstride; j += 32) sorted_out[(size_t)i * cstride + j] = j < nv ? S.ci[j] : kNone;
        if (lane == 0) out_cnt[i] = nr;
        __syncwarp();
    }
}

template <int NCH>
cudaError_t launch_acquire(const float *X, int64_t n, int d, const uint32_t *xs, int64_t nx, const uint32_t *cand,
                           int cstride, const int32_t *ncand, int M, int fill, uint32_t *out, int32_t *out_cnt,
                           uint32_t *sorted_out, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t want = (nx + kAcqWarps - 1) / kAcqWarps;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 16));
    acquire_kernel<NCH><<<(unsigned)blocks, 32 * kAcqWarps, 0, s>>>(X, n, d, xs, nx, cand, cstride, ncand, M, fill,
                                                                   out, out_cnt, sorted_out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t acquire_launch(const float *X, int64_t n, int d, const uint32_t *xs, int64_t nx, const uint32_t *cand,
                           int cstride, const int32_t *ncand, int M, int fill, uint32_t *out, int32_t *out_cnt,
                           uint32_t *sorted_out, cudaStream_t s) {
    switch (search_nch(d)) {
        case 1: return launch_acquire<1>(X, n, d, xs, nx, cand, cstride, ncand, M, fill, out, out_cnt, sorted_out, s);
        case 2: return launch_acquire<2>(X, n, d, xs, nx, cand, cstride, ncand, M, fill, out, out_cnt, sorted_out, s);
        case 4: return launch_acquire<4>(X, n, d, xs, nx, cand, cstride, ncand, M, fill, out, out_cnt, sorted_out, s);
        default: return launch_acquire<8>(X, n, d, xs, nx, cand, cstride, ncand, M, fill, out, out_cnt, sorted_out, s);
    }
}

}  // namespace roar

using namespace roar;

extern "C" roar_status roar_acquire(const float *X, int64_t n, int32_t d, const uint32_t *xs, int64_t nx,
                                    const uint32_t *cand, int32_t cand_stride, const int32_t *ncand, int32_t M,
                                    int32_t fill, uint32_t *out, int32_t *out_cnt, uint32_t *sorted_out,
                                    void *stream) {
    if (n < 1 || n >= (int64_t)kIdMask || d < 4 || d % 4 != 0 || d > 1024 || nx < 0 || M < 1 || M > kAcqMaxM ||
        cand_stride < 0 || cand_stride > kAcqMaxCand) {
        set_error("roar_acquire: need n >= 1, d % 4 == 0 and 4 <= d <= 1024, 1 <= M <= 64, "
                  "0 <= cand_stride <= 1024");
        return ROAR_EINVAL;
    }
    if (nx == 0) return ROAR_OK;
    if (!X || !xs || !ncand || !out || !out_cnt || (cand_stride > 0 && !cand) || !aligned(X, 16)) {
        set_error("roar_acquire: bad pointer (X must be 16-byte aligned)");
        return ROAR_EINVAL;
    }
    cudaError_t e = acquire_launch(X, n, d, xs, nx, cand, cand_stride, ncand, M, fill ? 1 : 0, out, out_cnt,
                                   sorted_out, (cudaStream_t)stream);
    return e == cudaSuccess ? ROAR_OK : cuda_fail(e, "roar_acquire");
}
