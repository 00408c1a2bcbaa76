// Beam-search kernels over BF16 traversal rows.
#include "roar_search_kernel.cuh"

namespace roar {
template const void *kernel_table<1>(int nch, int rpl, int tw, bool staged);
}  // namespace roar
