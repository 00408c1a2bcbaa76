// Beam-search kernels over F32 traversal rows (and the bipartite-graph search).
#include "roar_search_kernel.cuh"

namespace roar {
template const void *kernel_table<0>(int nch, int rpl, int tw, bool staged);
const void *kernel_table_bi(int nch, int rpl) { return kernel_table_bi_t<0>(nch, rpl); }
}  // namespace roar
