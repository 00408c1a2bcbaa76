// Beam-search kernels over FP8 traversal rows.
#include "roar_search_kernel.cuh"

namespace roar {
template const void *kernel_table<2>(int nch, int rpl, int tw, bool staged);
}  // namespace roar
