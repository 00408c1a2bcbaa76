// Beam-search dispatch: kernel choice, shared-memory sizing, occupancy and launch.
// The kernels themselves are in roar_search_kernel.cuh (one translation unit
// per traversal type).
#include "roar_internal.cuh"

namespace roar {

namespace {

int nch_for(int d) { return search_nch(d); }

int threads_for(int tw) { return 32 * (tw > kWarpsPerBlock ? tw : kWarpsPerBlock); }

}  // namespace

int teams_per_block(int tw) { return threads_for(tw) / (32 * tw); }

const void *search_kernel(int dtype, int d, int rmax, int tw, int lcap, bool bi = false) {
    const int nch = nch_for(d), rpl = rmax <= 64 ? 2 : 4;
    if (bi) return (dtype == 0 && tw == 1) ? kernel_table_bi(nch, rpl) : nullptr;
    const bool staged = search_staged(dtype, d, tw, lcap);
    switch (dtype) {
        case 0: return kernel_table<0>(nch, rpl, tw, staged);
        case 1: return kernel_table<1>(nch, rpl, tw, staged);
        case 2: return kernel_table<2>(nch, rpl, tw, staged);
        default: return nullptr;
    }
}

int hash_log2_for(int L) {
    // Measured on GB300 (1M x 200, 10k queries, FP32 / BF16 / FP8): the
    // global bitmap alone is faster from L = 20 on (15-20 % at L = 60-90); the
    // shared table only helps the shortest searches.
    if (L >= 16) return 0;
    const int lcap = (L + 31) / 32 * 32;
    const size_t budget = (size_t)(228 - kMinBlocksPerSm) * 1024;  // per SM, minus per-CTA reserve
    int lg = 10;
    while ((1 << lg) < 32 * L && lg < 14) ++lg;
    // Keep kMinBlocksPerSm CTAs resident; below 2^9 slots use the bitmap alone.
    while (lg >= 9 && search_smem_per_team(lcap, lg) * kWarpsPerBlock * kMinBlocksPerSm > budget) --lg;
    return lg >= 9 ? lg : 0;
}

int search_blocks_per_sm(int dtype, int d, int rmax, int lcap, int hash_log2, int tw, bool bi) {
    const void *fn = search_kernel(dtype, d, rmax, tw, lcap, bi);
    if (!fn) return 0;
    const size_t stage = bi ? 0 : search_stage_bytes(dtype, d, tw, lcap);
    const size_t smem = search_smem_per_team(lcap, hash_log2, stage) * teams_per_block(tw);
    if (smem > 227 * 1024) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, threads_for(tw), smem) != cudaSuccess)
        return 0;
    const int cap = kMaxWarpsPerSm * 32 / threads_for(tw);
    return blocks < cap ? blocks : cap;
}

cudaError_t launch_search(const SearchArgs &a, int blocks, int tw, cudaStream_t s, bool configure) {
    const bool bi = a.bi_off != nullptr;
    const void *fn = search_kernel(a.dtype, a.d, a.rmax, tw, a.lcap, bi);
    if (!fn || blocks <= 0) return cudaErrorInvalidValue;
    const size_t stage = bi ? 0 : search_stage_bytes(a.dtype, a.d, tw, a.lcap);
    const size_t smem = search_smem_per_team(a.lcap, a.hash_log2, stage) * teams_per_block(tw);
    cudaError_t e = cudaSuccess;
    if (configure) {  // already done by search_blocks_per_sm when planning
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemsetAsync(a.work, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<SearchArgs *>(&a)};
    return cudaLaunchKernel(fn, dim3(blocks), dim3(threads_for(tw)), args, smem, s);
}

}  // namespace roar
