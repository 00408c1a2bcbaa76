// Dense steps: reduced-precision copies of the base rows, and the exact
// k-nearest-neighbour search of many queries against the base set, which is
// the preprocessing step of RoarGraph's construction ("ground truths of the
// training queries", Sec. 4.2.1) and also yields the evaluation ground truth
// (Sec. 2.1.1).
//
// kNN pipeline per block of R query rows:
//   1. S = Tq . Xq^T on the tensor cores (BF16 inputs, FP32 accumulation);
//   2. one warp per row keeps a running top-C list of S's row under
//      (distance = -score, id) in shared memory; a column enters only if it
//      beats the current C-th entry, so after the first few thousand columns
//      almost every column is rejected by one compare;
//   3. the C candidates are re-scored with exact FP32 dot products (the
//      search's fixed order) and the first kk in (distance, id) order are kept.
// With C > kk the BF16 rounding of step 1 only has to keep the true top-kk
// inside the top-C, which a margin of C - kk ranks makes near-certain; the
// returned distances are exact FP32 values.
#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
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

// Running top-C per row of a score block S [R][ldS] (scores = <t, x>), columns
// [0, ncols) map to ids col0 + c. One warp per row; the list lives in shared
// memory sorted by (-score, id). Writes ids/dist [R][C] (dist = -score).
template <int C>
__global__ void __launch_bounds__(256) topk_rows_kernel(const float *__restrict__ S, int64_t R,
                                                        int64_t ncols, int64_t ldS, uint32_t col0,
                                                        uint32_t *__restrict__ out_ids,
                                                        float *__restrict__ out_d) {
    __shared__ float sd[8][C];
    __shared__ uint32_t si[8][C];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + w;
    if (row >= R) return;
    float *kd = sd[w];
    uint32_t *ki = si[w];
    const float *srow = S + row * ldS;
    int size = 0;
    float wd = __int_as_float(0x7f800000);   // current worst kept distance (+inf while not full)
    uint32_t wi = 0xFFFFFFFFu;
    for (int64_t base = 0; base < ncols; base += 128) {
        float dv[4];
        uint32_t iv[4];
        const int64_t c0 = base + lane * 4;
        if (c0 + 3 < ncols && (ldS % 4) == 0) {
            const float4 v = __ldcs(reinterpret_cast<const float4 *>(srow + c0));
            dv[0] = -v.x; dv[1] = -v.y; dv[2] = -v.z; dv[3] = -v.w;
        } else {
#pragma unroll
            for (int t = 0; t < 4; ++t)
                dv[t] = (c0 + t < ncols) ? -srow[c0 + t] : __int_as_float(0x7f800000);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) iv[t] = col0 + (uint32_t)(c0 + t);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const bool valid = c0 + t < ncols;
            unsigned m = __ballot_sync(kFull, valid && (size < C || less_entry(dv[t], iv[t], wd, wi)));
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1;
                const float dd = __shfl_sync(kFull, dv[t], src);
                const uint32_t ii = __shfl_sync(kFull, iv[t], src);
                if (size == C && !less_entry(dd, ii, wd, wi)) continue;
                // insertion position = number of kept entries before (dd, ii)
                int pos = 0;
#pragma unroll
                for (int j = 0; j < C / 32; ++j) {
                    const int e = lane + 32 * j;
                    const bool before = e < size && less_entry(kd[e], ki[e], dd, ii);
                    pos += __popc(__ballot_sync(kFull, before));
                }
                // shift [pos, size) right by one (the last falls off when full)
                float mvd[C / 32];
                uint32_t mvi[C / 32];
#pragma unroll
                for (int j = 0; j < C / 32; ++j) {
                    const int e = lane + 32 * j;
                    if (e >= pos && e < size) {
                        mvd[j] = kd[e];
                        mvi[j] = ki[e];
                    }
                }
                __syncwarp();
#pragma unroll
                for (int j = 0; j < C / 32; ++j) {
                    const int e = lane + 32 * j;
                    if (e >= pos && e < size && e + 1 < C) {
                        kd[e + 1] = mvd[j];
                        ki[e + 1] = mvi[j];
                    }
                }
                if (lane == 0) {
                    kd[pos] = dd;
                    ki[pos] = ii;
                }
                __syncwarp();
                if (size < C) ++size;
                if (size == C) {
                    wd = kd[C - 1];
                    wi = ki[C - 1];
                }
            }
        }
    }
    for (int j = lane; j < C; j += 32) {
        out_ids[row * C + j] = j < size ? ki[j] : 0xFFFFFFFFu;
        out_d[row * C + j] = j < size ? kd[j] : __int_as_float(0x7f800000);
    }
}

// Merge two sorted (dist, id) lists of length C per row (running result and a
// new column block's result) into the first C of their union.
template <int C>
__global__ void merge_lists_kernel(int64_t R, uint32_t *__restrict__ acc_i, float *__restrict__ acc_d,
                                   const uint32_t *__restrict__ new_i, const float *__restrict__ new_d) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= R) return;
    uint32_t *ai = acc_i + row * C;
    float *ad = acc_d + row * C;
    const uint32_t *bi = new_i + row * C;
    const float *bd = new_d + row * C;
    float od[C / 32];
    uint32_t oi[C / 32];
    int op[C / 32];
    float nd[C / 32];
    uint32_t ni[C / 32];
    int np[C / 32];
#pragma unroll
    for (int j = 0; j < C / 32; ++j) {
        const int e = lane + 32 * j;
        od[j] = ad[e];
        oi[j] = ai[e];
        nd[j] = bd[e];
        ni[j] = bi[e];
        // rank of each element in the union: own index + elements of the other list before it
        int lo = 0, hi = C;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (less_entry(bd[mid], bi[mid], od[j], oi[j])) lo = mid + 1; else hi = mid;
        }
        op[j] = e + lo;
        lo = 0;
        hi = C;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (less_entry(ad[mid], ai[mid], nd[j], ni[j])) lo = mid + 1; else hi = mid;
        }
        np[j] = e + lo;
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < C / 32; ++j) {
        if (op[j] < C) { ad[op[j]] = od[j]; ai[op[j]] = oi[j]; }
        if (np[j] < C) { ad[np[j]] = nd[j]; ai[np[j]] = ni[j]; }
    }
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
    const int d4 = d >> 2;
    const float4 *q4 = reinterpret_cast<const float4 *>(T + row * d);
    for (int j = 0; j < C; ++j) {
        const uint32_t u = cand[row * C + j];
        float s = 0.0f;
        if (u != 0xFFFFFFFFu) {
            const float4 *x4 = reinterpret_cast<const float4 *>(X + (int64_t)u * d);
            for (int ch = lane; ch < d4; ch += 32) {
                const float4 a = __ldg(q4 + ch), b = __ldg(x4 + ch);
                s = fmaf(a.x, b.x, s);
                s = fmaf(a.y, b.y, s);
                s = fmaf(a.z, b.z, s);
                s = fmaf(a.w, b.w, s);
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s = s + __shfl_xor_sync(kFull, s, o);
        if (lane == 0) {
            sd[w][j] = (u != 0xFFFFFFFFu) ? -s : __int_as_float(0x7f800000);
            si[w][j] = u;
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

roar_status quantize_bf16(const float *X, int64_t n, int d, void *out, cudaStream_t s) {
    const int64_t blocks = (n + 7) / 8;
    quantize_bf16_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, n, d, (__nv_bfloat16 *)out);
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

namespace {
const char *cublas_name(cublasStatus_t st) {
    switch (st) {
        case CUBLAS_STATUS_SUCCESS: return "success";
        case CUBLAS_STATUS_NOT_INITIALIZED: return "not initialized";
        case CUBLAS_STATUS_ALLOC_FAILED: return "alloc failed";
        case CUBLAS_STATUS_INVALID_VALUE: return "invalid value";
        case CUBLAS_STATUS_EXECUTION_FAILED: return "execution failed";
        default: return "error";
    }
}
}  // namespace

extern "C" roar_status roar_knn(const float *T, int64_t nt, const float *X, int64_t n, int32_t d,
                                int32_t kk, uint32_t *ids, float *dist, void *stream) {
    constexpr int C = 128;
    if (nt < 0 || n < 1 || n >= 0x7FFFFFFF || d < 4 || d % 4 != 0 || d > 1024 || kk < 1 ||
        kk > C || kk > n) {
        set_error("roar_knn: need n >= kk, 1 <= kk <= 128, d % 4 == 0, d <= 1024");
        return ROAR_EINVAL;
    }
    if (nt == 0) return ROAR_OK;
    if (!T || !X || !ids || !dist || !aligned(T, 16) || !aligned(X, 16)) return ROAR_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // Column blocks keep the score block under ~8 GB; row blocks of 4096 queries.
    const int64_t RB = std::min<int64_t>(nt, 4096);
    const int64_t CB = std::min<int64_t>(n, (int64_t)1 << 19);
    __nv_bfloat16 *t16 = nullptr, *x16 = nullptr;
    float *S = nullptr, *cd = nullptr, *nd = nullptr;
    uint32_t *ci = nullptr, *ni = nullptr;
    cublasHandle_t h = nullptr;
    roar_status rc = ROAR_OK;
    cudaError_t e = cudaMalloc(&t16, (size_t)nt * d * 2);
    if (e == cudaSuccess) e = cudaMalloc(&x16, (size_t)n * d * 2);
    if (e == cudaSuccess) e = cudaMalloc(&S, (size_t)RB * CB * 4);
    if (e == cudaSuccess) e = cudaMalloc(&ci, (size_t)RB * C * 4);
    if (e == cudaSuccess) e = cudaMalloc(&cd, (size_t)RB * C * 4);
    if (e == cudaSuccess) e = cudaMalloc(&ni, (size_t)RB * C * 4);
    if (e == cudaSuccess) e = cudaMalloc(&nd, (size_t)RB * C * 4);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("roar_knn: out of device memory");
        rc = ROAR_ENOMEM;
        goto done;
    }
    if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS || cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) {
        set_error("roar_knn: cublasCreate failed");
        rc = ROAR_ECUDA;
        goto done;
    }
    if ((rc = quantize_bf16(T, nt, d, t16, s)) != ROAR_OK) goto done;
    if ((rc = quantize_bf16(X, n, d, x16, s)) != ROAR_OK) goto done;
    for (int64_t r0 = 0; r0 < nt; r0 += RB) {
        const int64_t rb = std::min(RB, nt - r0);
        for (int64_t c0 = 0; c0 < n; c0 += CB) {
            const int64_t cb = std::min(CB, n - c0);
            const float one = 1.0f, zero = 0.0f;
            // column-major view: S^T (cb x rb) = X_blk (cb x d) . T_blk^T (d x rb), ld = cb
            cublasStatus_t cs = cublasGemmEx(h, CUBLAS_OP_T, CUBLAS_OP_N, (int)cb, (int)rb, d, &one,
                                             x16 + c0 * d, CUDA_R_16BF, d, t16 + r0 * d, CUDA_R_16BF,
                                             d, &zero, S, CUDA_R_32F, (int)cb, CUBLAS_COMPUTE_32F,
                                             CUBLAS_GEMM_DEFAULT);
            if (cs != CUBLAS_STATUS_SUCCESS) {
                char msg[96];
                std::snprintf(msg, sizeof msg, "roar_knn: cublasGemmEx %s", cublas_name(cs));
                set_error(msg);
                rc = ROAR_ECUDA;
                goto done;
            }
            uint32_t *dst_i = c0 == 0 ? ci : ni;
            float *dst_d = c0 == 0 ? cd : nd;
            topk_rows_kernel<C><<<(unsigned)((rb + 7) / 8), 256, 0, s>>>(S, rb, cb, cb, (uint32_t)c0,
                                                                      dst_i, dst_d);
            if (c0 != 0)
                merge_lists_kernel<C><<<(unsigned)((rb + 7) / 8), 256, 0, s>>>(rb, ci, cd, ni, nd);
        }
        rescore_kernel<C><<<(unsigned)((rb + 3) / 4), 128, 0, s>>>(T + r0 * d, rb, X, d, ci, kk,
                                                                 ids + r0 * kk, dist + r0 * kk);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "roar_knn kernels");
            goto done;
        }
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "roar_knn");
done:
    if (h) cublasDestroy(h);
    cudaFree(t16);
    cudaFree(x16);
    cudaFree(S);
    cudaFree(ci);
    cudaFree(cd);
    cudaFree(ni);
    cudaFree(nd);
    return rc;
}
