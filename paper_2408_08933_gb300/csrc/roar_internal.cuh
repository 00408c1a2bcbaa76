// Internal declarations shared by the CUDA translation units of libroargraph.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "roargraph.h"

namespace roar {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kChecked = 0x80000000u;   // pool entry already expanded
constexpr uint32_t kIdMask = 0x7FFFFFFFu;
constexpr int kWarpsPerBlock = 4;            // one query per warp, 4 per CTA
constexpr int kCandCap = ROAR_MAX_RMAX;      // new neighbours per hop, at most rmax
constexpr int kMaxWarpsPerSm = 32;
#ifndef ROAR_MIN_BLOCKS
#define ROAR_MIN_BLOCKS 4
#endif
constexpr int kMinBlocksPerSm = ROAR_MIN_BLOCKS;  // register budget: 65536 / (blocks * 128)
// The BF16 / FP8 traversal kernels hold narrower row chunks and are compiled
// for more resident CTAs: measured on GB300 (1M x 200, L = 20-300), 6 CTAs per
// SM for BF16 and 8 for FP8 were fastest despite a few hundred bytes of spills.
#ifndef ROAR_MIN_BLOCKS_BF16
#define ROAR_MIN_BLOCKS_BF16 6
#endif
#ifndef ROAR_MIN_BLOCKS_FP8
#define ROAR_MIN_BLOCKS_FP8 8
#endif
// For wide rows (NCH >= 4 chunks per lane, d > 256) the BF16 / FP8 kernels
// hold four query chunks per lane and run best with the full 128-register
// budget of 4 CTAs per SM (measured on GB300, 1M x 512: 20-25 % faster than
// 6 or 8 CTAs at L = 100-400).
#ifndef ROAR_MIN_BLOCKS_LOWP_WIDE
#define ROAR_MIN_BLOCKS_LOWP_WIDE 4
#endif
template <int DT, int NCH = 1>
__host__ __device__ constexpr int min_blocks_per_sm() {
    return DT == 0 ? ROAR_MIN_BLOCKS
                   : (NCH >= 4 ? ROAR_MIN_BLOCKS_LOWP_WIDE : (DT == 1 ? ROAR_MIN_BLOCKS_BF16 : ROAR_MIN_BLOCKS_FP8));
}
#define ROAR_NOALLOC_SCRATCH_BYTES (64ull << 20)

// Everything one search launch needs. Plain pointers: the launch reads the
// index rows, the queries and the scratch, and writes the result arrays.
struct SearchArgs {
    const void *trav;        // traversal rows: FP32, BF16 or FP8 [n][d]
    const float *scales;     // FP8 per-row scales [n] or null
    const float *base32;     // FP32 rows [n][d] (re-rank)
    const uint32_t *adj;     // [n][rmax]
    const uint32_t *tomb;    // deletion bitmap [ceil(n/32)] or null: deleted rows route, are not answers
    int64_t n;
    int32_t d;
    int32_t rmax;
    uint32_t entry;
    int32_t dtype;           // roar_dtype of `trav`
    const float *q;          // [nq][d]
    int64_t nq;
    int32_t k, L;            // uniform k and L ...
    const int32_t *k_arr;    // ... or per query (uneven batches)
    const int32_t *L_arr;
    const int64_t *out_off;  // per-query first result slot (uneven batches)
    const int32_t *order;    // optional processing order (a permutation of 0..nq-1)
    int32_t lcap;            // pool capacity, multiple of 32, >= every L
    uint32_t max_visits;
    int32_t hash_log2;       // shared-memory visited-table slots, log2 (0: none)
    uint32_t *vbits;         // per-warp-slot visited bitmaps, vbits_words each, all-zero at rest
    int64_t vbits_words;
    uint32_t *vlog;          // per-warp-slot log of the ids set in the bitmap, vlog_cap each
    int32_t vlog_cap;
    unsigned int *work;      // next unclaimed query (reset per launch)
    // Serving ring in device memory (all null for batch launches): queries,
    // k, L and result slots are indexed by slot = sequence % ring_cap.
    const float *ring_rec;                         // per slot: query (d floats), k, L (int32), padding
    int32_t ring_stride;                           // floats per record (a multiple of 4)
    const uint32_t *ring_pub;                      // per slot, low 32 bits of seq + 1 once published
    unsigned long long *ring_head;                 // tickets taken so far
    unsigned long long *ring_orphan;               // per team slot: a ticket kept over an idle exit, or ~0
    volatile uint32_t *ring_done;                  // per slot, low 32 bits of seq + 1 when done
    const volatile int *ring_stop;                 // nonzero asks the kernel to exit
    int64_t ring_cap;
    int32_t ring_kmax;                             // result slots per ring entry
    uint32_t idle_polls;                           // microseconds without a served ticket before the kernel exits
    unsigned long long *ring_clock;                // [0] global time of the last ticket served, [1] closing flag
    uint32_t *ids;
    float *dist;
    uint32_t *visits;
    uint32_t *hops;
    int32_t *qstatus;
    // Bipartite graph G_bi (null for a plain graph): expanding base node v
    // scans, for each query node t in B(v) = bi_q[bi_off[v] .. bi_off[v+1]),
    // the row t of `adj`, which then holds N_out(t) for bi_nt query nodes.
    const int64_t *bi_off;
    const uint32_t *bi_q;
    int64_t bi_nt;
    // Optional expansion trace (batch launches, null otherwise): the first
    // trace_cap nodes a query expands, in order, at trace[qi * trace_cap ..];
    // `hops` tells how many there were. trace_bound (optional) gets, for each,
    // the pool's L-th distance when it was expanded (+inf while not full).
    uint32_t *trace;
    float *trace_bound;
    int32_t trace_cap;
};

// Shared memory of one warp: pool (8 B per slot), candidate buffers (16 B per
// slot), optional visited table (4 B per slot).
__host__ __device__ inline size_t search_smem_per_warp(int lcap, int hash_log2) {
    return (size_t)lcap * 8 + (size_t)kCandCap * 16 + (hash_log2 ? ((size_t)4 << hash_log2) : 0);
}

// 16-byte row chunks a lane holds: rows of d floats are d/4 chunks dealt to
// 32 lanes, NCH = 1, 2, 4 or 8 per lane.
__host__ __device__ inline int search_nch(int d) {
    const int need = ((d >> 2) + 31) / 32;
    return need <= 1 ? 1 : need <= 2 ? 2 : need <= 4 ? 4 : 8;
}

// For short searches the one-warp kernels can stage their row gathers in
// shared memory: two buffers of stage_rows(dtype, NCH) rows per warp (FP32:
// ROAR_STAGE_ROWS rows for d <= 256, BF16 / FP8: ROAR_STAGE_ROWS_LOWP;
// proportionally fewer for wider rows). Measured on GB300 (1M x 200), FP32
// with 4 rows: 3-8 % faster at L = 50-150 and equal at L = 300; for longer
// pools the extra shared memory costs more occupancy than it gains, so the
// staged variants run only while lcap <= ROAR_STAGE_MAX_LCAP.
#ifndef ROAR_STAGE_ROWS
#define ROAR_STAGE_ROWS 4
#endif
// BF16 / FP8 staging is off by default: on GB300 (1M x 200, L = 50-300) it was
// 5-30 % slower than their register path, which already gathers 8 rows per batch.
#ifndef ROAR_STAGE_ROWS_LOWP
#define ROAR_STAGE_ROWS_LOWP 0
#endif
#ifndef ROAR_STAGE_MAX_LCAP
#define ROAR_STAGE_MAX_LCAP 320
#endif
// Register budget of the staged FP32 kernel, in 4-warp CTAs per SM: 5 (96
// registers, no spills) measured 3.5 % faster at L = 90 than 4, 6 and 8.
#ifndef ROAR_MIN_BLOCKS_STAGED
#define ROAR_MIN_BLOCKS_STAGED 5
#endif
// Bytes of one 4-element row chunk: FP32 16, BF16 8, FP8 4.
__host__ __device__ constexpr int chunk_bytes(int dtype) { return 16 >> dtype; }
__host__ __device__ constexpr int stage_rows(int dtype, int nch) {
    return (dtype == 0 ? ROAR_STAGE_ROWS : ROAR_STAGE_ROWS_LOWP) <= 0 ? 0
           : nch <= 2 ? (dtype == 0 ? ROAR_STAGE_ROWS : ROAR_STAGE_ROWS_LOWP)
           : ((dtype == 0 ? ROAR_STAGE_ROWS : ROAR_STAGE_ROWS_LOWP) * 2 / nch > 0
                  ? (dtype == 0 ? ROAR_STAGE_ROWS : ROAR_STAGE_ROWS_LOWP) * 2 / nch
                  : 1);
}
// Staging bytes per warp for S rows per buffer: two buffers of S rows of d4
// chunks, then (FP8) two buffers of S row scales; a multiple of 16.
__host__ __device__ inline size_t stage_bytes(int dtype, int S, int d4) {
    const size_t b = (size_t)2 * S * d4 * chunk_bytes(dtype) + (dtype == 2 ? (size_t)2 * S * 4 : 0);
    return (b + 15) / 16 * 16;
}
// Rows are copied in 16-byte pieces, so a row's bytes must be a multiple of 16
// (FP32: any d % 4 == 0; BF16: d % 8 == 0; FP8: d % 16 == 0).
__host__ __device__ inline bool search_staged(int dtype, int d, int tw, int lcap) {
    return tw == 1 && lcap <= ROAR_STAGE_MAX_LCAP && stage_rows(dtype, 1) > 0 &&
           ((size_t)d * (4 >> dtype)) % 16 == 0;
}
__host__ __device__ inline size_t search_stage_bytes(int dtype, int d, int tw, int lcap) {
    if (!search_staged(dtype, d, tw, lcap)) return 0;
    return stage_bytes(dtype, stage_rows(dtype, search_nch(d)), d >> 2);
}

// Per team: the above plus a 16-byte control block (claimed query, hop count,
// pool size), then `stage` bytes of gather staging.
__host__ __device__ inline size_t search_smem_per_team(int lcap, int hash_log2, size_t stage = 0) {
    return search_smem_per_warp(lcap, hash_log2) + 16 + stage;
}
// Resident CTAs per SM for this configuration with teams of tw warps (0 if it
// cannot launch), the teams per CTA, and the launch itself.
int search_blocks_per_sm(int dtype, int d, int rmax, int lcap, int hash_log2, int tw, bool bi = false);
int teams_per_block(int tw);
cudaError_t launch_search(const SearchArgs &a, int blocks, int tw, cudaStream_t s, bool configure = true);
template <int DT>
const void *kernel_table(int nch, int rpl, int tw, bool staged);
const void *kernel_table_bi(int nch, int rpl);

int hash_log2_for(int L);

// Fills a SearchArgs for a handle (index rows, tuning, scratch sized for the
// full resident grid) and picks blocks and team warps. Defined in roar_capi.cu.
roar_status plan_search(roar_index *idx, int32_t lmax, SearchArgs &a, int &blocks, int &tw, int64_t nq);

}  // namespace roar
