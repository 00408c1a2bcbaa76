// The query-base bipartite graph G_bi of Alg. 1 (Sec. 4.2.2), laid out for
// the search kernel's bipartite mode: B(x) as CSR (offsets per base node,
// query ids ascending) and the N_out rows of the query nodes.
#include <cuda_runtime.h>

#include <cstdio>
#include <vector>

#include "roargraph.h"

namespace roar {
roar_status cuda_fail(cudaError_t e, const char *what);
void set_error(const char *msg);
}  // namespace roar

using namespace roar;

extern "C" roar_status roar_bipartite(const uint32_t *knn, int64_t nt, int32_t nqd, int64_t n, int64_t *off,
                                      uint32_t *qids, uint32_t *nout, int64_t *stats, void *stream) {
    if (!knn || !off || !qids || !nout || nt < 1 || nt >= ((int64_t)1 << 31) || n < 1 || n >= ((int64_t)1 << 31) ||
        nqd < 2 || nqd - 1 > ROAR_MAX_RMAX) {
        set_error("roar_bipartite: need nt >= 1, n >= 1, 2 <= nqd <= ROAR_MAX_RMAX + 1 and non-null arrays");
        return ROAR_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // Each training query's nearest base row (rank 0 of its kNN list).
    std::vector<uint32_t> piv((size_t)nt);
    cudaError_t e = cudaMemcpy2DAsync(piv.data(), sizeof(uint32_t), knn, (size_t)nqd * sizeof(uint32_t),
                                      sizeof(uint32_t), (size_t)nt, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "roar_bipartite: pivots");
    // x -> t for every t whose nearest base row is x: counting sort, t ascending.
    std::vector<int64_t> o((size_t)n + 1, 0);
    for (int64_t t = 0; t < nt; ++t) {
        if ((int64_t)piv[(size_t)t] >= n) {
            set_error("roar_bipartite: a kNN id is not below n");
            return ROAR_EINVAL;
        }
        ++o[(size_t)piv[(size_t)t] + 1];
    }
    int64_t pivots = 0, widest = 0;
    for (int64_t x = 0; x < n; ++x) {
        pivots += o[(size_t)x + 1] > 0;
        if (o[(size_t)x + 1] > widest) widest = o[(size_t)x + 1];
        o[(size_t)x + 1] += o[(size_t)x];
    }
    std::vector<int64_t> fill(o.begin(), o.end() - 1);
    std::vector<uint32_t> q((size_t)nt);
    for (int64_t t = 0; t < nt; ++t) q[(size_t)fill[piv[(size_t)t]]++] = (uint32_t)t;
    e = cudaMemcpyAsync(off, o.data(), o.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(qids, q.data(), q.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    // N_out(t): the kNN list without its rank-0 entry (the edge t -> x removed).
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(nout, (size_t)(nqd - 1) * sizeof(uint32_t), knn + 1, (size_t)nqd * sizeof(uint32_t),
                              (size_t)(nqd - 1) * sizeof(uint32_t), (size_t)nt, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "roar_bipartite: upload");
    if (stats) {
        stats[0] = pivots;
        stats[1] = widest;
    }
    return ROAR_OK;
}
