// Beam-search kernels over F32 traversal rows.
#include "roar_search_kernel.cuh"

namespace roar {
template const void *kernel_table<0>(int nch, int rpl, int tw, bool staged);
}  // namespace roar
