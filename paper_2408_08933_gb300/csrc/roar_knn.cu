// Dense steps: reduced-precision copies of the base rows, and the exact
// k-nearest-neighbour search of many queries against the base set, which is
// the preprocessing step of RoarGraph's construction ("ground truths of the
// training queries", Sec. 4.2.1) and also yields the evaluation ground truth
// (Sec. 2.1.1).
//
// kNN pipeline per block of query rows:
//   1. BF16 copies of both sides (round to nearest even);
//   2. scores on the 5th-generation tensor cores with a fused running top-C
//      per row (roar_knn_tc.cu): no score matrix is written;
//   3. the C candidates are re-scored with exact FP32 dot products (the
//      search's fixed order) and the first kk in (distance, id) order are kept.
// With C > kk the BF16 rounding of step 2 only has to keep the true top-kk
// inside the top-C, which a margin of C - kk ranks makes near-certain; the
// returned distances are exact FP32 values.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <atomic>
#include <cstdio>

#include "roar_internal.cuh"

namespace roar {

roar_status cuda_fail(cudaError_t e, const char *what);
void set_error(const char *msg);
bool aligned(const void *p, size_t a);

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ bool less_entry(float da, uint32_t ia, float db, uint32_t ib) {
    return da < db || (da == db && ia < ib);
}

// One warp per row. BF16: round to nearest even, scale 1.
__global__ void quantize_bf16_kernel(const float *__restrict__ X, int64_t n, int d,
                                     __nv_bfloat16 *__restrict__ out) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const float *x = X + row * d;
    __nv_bfloat16 *o = out + row * d;
    for (int i = lane; i < d; i += 32) o[i] = __float2bfloat16_rn(x[i]);
}

// One warp per row: BF16 rows padded with zeros to dp columns (the kNN
// kernel's operands: rows of whole 64-column K chunks, so each chunk of a row
// is one aligned 128-byte segment).
__global__ void quantize_bf16_pad_kernel(const float *__restrict__ X, int64_t n, int d, int dp,
                                         __nv_bfloat16 *__restrict__ out) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const float *x = X + row * d;
    __nv_bfloat16 *o = out + row * dp;
    for (int i = lane; i < dp; i += 32) o[i] = i < d ? __float2bfloat16_rn(x[i]) : __float2bfloat16_rn(0.0f);
}

// One warp per row. FP8-E4M3: s = maxabs / 448 (IEEE division), code = E4M3(x / s)
// rounded to nearest even and saturated to +-448; an all-zero row gets s = 1.
__global__ void quantize_fp8_kernel(const float *__restrict__ X, int64_t n, int d,
                                    uint8_t *__restrict__ out, float *__restrict__ scales) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const float *x = X + row * d;
    float m = 0.0f;
    for (int i = lane; i < d; i += 32) m = fmaxf(m, fabsf(x[i]));
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    const float s = (m == 0.0f) ? 1.0f : __fdiv_rn(m, 448.0f);
    if (lane == 0) scales[row] = s;
    uint8_t *o = out + row * d;
    for (int i = lane; i < d; i += 32)
        o[i] = (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(x[i], s), __NV_SATFINITE, __NV_E4M3);
}

// Exact FP32 re-scoring of C candidates per query row, then the first kk in
// (distance, id) order. One warp per row; dot products use the fixed order
// (element i on lane (i >> 2) & 31, fmaf, xor butterfly).
template <int C>
__global__ void rescore_kernel(const float *__restrict__ T, int64_t nt, const float *__restrict__ X,
                               int d, const uint32_t *__restrict__ cand, int kk,
                               uint32_t *__restrict__ ids, float *__restrict__ dist) {
    __shared__ float sd[4][C];
    __shared__ uint32_t si[4][C];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 4 + w;
    if (row >= nt) return;
    const int d4 = d >> 2;   // d <= 512: at most 4 chunks per lane
    const float4 *q4 = reinterpret_cast<const float4 *>(T + row * d);
    float4 qv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int ch = lane + 32 * c;
        qv[c] = ch < d4 ? __ldg(q4 + ch) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // G candidates at a time, so that their row loads are in flight together;
    // each candidate's sum keeps its own order (chunks in increasing index).
    constexpr int G = 4;
    static_assert(C % G == 0, "candidates come in groups of G");
    for (int j0 = 0; j0 < C; j0 += G) {
        uint32_t u[G];
        float s[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            u[g] = cand[row * C + j0 + g];
            s[g] = 0.0f;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int ch = lane + 32 * c;
            if (ch >= d4) break;
            float4 b[G];
#pragma unroll
            for (int g = 0; g < G; ++g)
                b[g] = u[g] != 0xFFFFFFFFu ? __ldg(reinterpret_cast<const float4 *>(X + (int64_t)u[g] * d) + ch)
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                s[g] = fmaf(qv[c].x, b[g].x, s[g]);
                s[g] = fmaf(qv[c].y, b[g].y, s[g]);
                s[g] = fmaf(qv[c].z, b[g].z, s[g]);
                s[g] = fmaf(qv[c].w, b[g].w, s[g]);
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) s[g] = s[g] + __shfl_xor_sync(kFull, s[g], o);
            if (lane == 0) {
                sd[w][j0 + g] = (u[g] != 0xFFFFFFFFu) ? -s[g] : __int_as_float(0x7f800000);
                si[w][j0 + g] = u[g];
            }
        }
    }
    __syncwarp();
    for (int j = lane; j < C; j += 32) {
        const float dj = sd[w][j];
        const uint32_t ij = si[w][j];
        int r = 0;
        for (int x = 0; x < C; ++x) r += less_entry(sd[w][x], si[w][x], dj, ij) ? 1 : 0;
        if (r < kk) {
            ids[row * kk + r] = ij;
            dist[row * kk + r] = dj;
        }
    }
}

}  // namespace

roar_status quantize_bf16_pad(const float *X, int64_t n, int d, int dp, void *out, cudaStream_t s) {
    const int64_t blocks = (n + 7) / 8;
    quantize_bf16_pad_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, n, d, dp, (__nv_bfloat16 *)out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ROAR_OK : cuda_fail(e, "quantize_bf16");
}

}  // namespace roar

using namespace roar;

extern "C" roar_status roar_quantize(const float *X, int64_t n, int32_t d, roar_dtype dtype,
                                     void *out, float *scales, void *stream) {
    if (n < 0 || d < 4 || d % 4 != 0 || d > 1024) return ROAR_EINVAL;
    if (n == 0) return ROAR_OK;
    if (!X || !out) return ROAR_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t blocks = (n + 7) / 8;
    if (blocks > 0x7FFFFFFF) return ROAR_EINVAL;
    if (dtype == ROAR_BF16) {
        quantize_bf16_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, n, d, (__nv_bfloat16 *)out);
    } else if (dtype == ROAR_FP8_E4M3) {
        if (!scales) return ROAR_EINVAL;
        quantize_fp8_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, n, d, (uint8_t *)out, scales);
    } else {
        return ROAR_EINVAL;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ROAR_OK : cuda_fail(e, "roar_quantize");
}

namespace roar {
cudaError_t knn_tc_launch(const __nv_bfloat16 *T16, int64_t nt, const __nv_bfloat16 *X16, int64_t n, int d,
                          int C, int cap, float *buf_s, uint32_t *buf_i, uint32_t *cand, int *err,
                          uint64_t wait_ns, cudaStream_t s);
int64_t knn_tc_wave_rows(int d);
// Wall-time limit of each bounded wait in the tensor-core kernel: 2 s by
// default, far above any legitimate wait there.
constexpr int64_t kKnnWaitDefaultNs = 2000000000ll;
static std::atomic<int64_t> g_knn_wait_ns{kKnnWaitDefaultNs};
}  // namespace roar

extern "C" roar_status roar_knn_set_wait_limit_ns(int64_t ns) {
    g_knn_wait_ns.store(ns < 0 ? kKnnWaitDefaultNs : ns);
    return ROAR_OK;
}

extern "C" roar_status roar_knn(const float *T, int64_t nt, const float *X, int64_t n, int32_t d,
                                int32_t kk, uint32_t *ids, float *dist, void *stream) {
    constexpr int C = 128, CAP = 1024;
    if (nt < 0 || n < 1 || n >= 0x7FFFFFFF || d < 8 || d % 8 != 0 || d > 512 || kk < 1 || kk > C ||
        kk > n) {
        set_error("roar_knn: need n >= kk, 1 <= kk <= 128, d % 8 == 0, 8 <= d <= 512");
        return ROAR_EINVAL;
    }
    if (nt == 0) return ROAR_OK;
    if (!T || !X || !ids || !dist || !aligned(T, 16) || !aligned(X, 16)) return ROAR_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int dp = (d + 63) / 64 * 64;   // BF16 operand rows padded to whole 64-column K chunks
    // Query rows per launch: whole waves of the kernel, about 131,072 at most
    // (a partial last wave leaves SMs idle for a whole sweep of X).
    const int64_t wave = knn_tc_wave_rows(dp);
    const int64_t RB = std::min<int64_t>(nt, std::max<int64_t>(wave, 131072 / wave * wave));
    __nv_bfloat16 *t16 = nullptr, *x16 = nullptr;
    float *bs = nullptr;
    uint32_t *bi = nullptr, *cand = nullptr;
    int *err = nullptr;
    const uint64_t wait_ns = (uint64_t)g_knn_wait_ns.load();
    roar_status rc = ROAR_OK;
    int herr = 0;
    cudaError_t e = cudaMalloc(&t16, (size_t)nt * dp * 2);
    if (e == cudaSuccess) e = cudaMalloc(&x16, (size_t)n * dp * 2);
    if (e == cudaSuccess) e = cudaMalloc(&bs, (size_t)RB * CAP * 4);
    if (e == cudaSuccess) e = cudaMalloc(&bi, (size_t)RB * CAP * 4);
    if (e == cudaSuccess) e = cudaMalloc(&cand, (size_t)RB * C * 4);
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("roar_knn: out of device memory");
        rc = ROAR_ENOMEM;
        goto done;
    }
    if ((rc = quantize_bf16_pad(T, nt, d, dp, t16, s)) != ROAR_OK) goto done;
    if ((rc = quantize_bf16_pad(X, n, d, dp, x16, s)) != ROAR_OK) goto done;
    for (int64_t r0 = 0; r0 < nt; r0 += RB) {
        const int64_t rb = std::min(RB, nt - r0);
        e = knn_tc_launch(t16 + r0 * dp, rb, x16, n, dp, C, CAP, bs, bi, cand, err, wait_ns, s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "roar_knn: tensor-core scores");
            goto done;
        }
        rescore_kernel<C><<<(unsigned)((rb + 3) / 4), 128, 0, s>>>(T + r0 * d, rb, X, d, cand, kk,
                                                                 ids + r0 * kk, dist + r0 * kk);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "roar_knn: rescore");
            goto done;
        }
    }
    e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "roar_knn");
    else if (herr) {
        set_error("roar_knn: a tensor-core wait timed out");
        rc = ROAR_ETIMEOUT;
    }
done:
    cudaFree(t16);
    cudaFree(x16);
    cudaFree(bs);
    cudaFree(bi);
    cudaFree(cand);
    cudaFree(err);
    return rc;
}
