// Pass kernels for lines of 8 nodes, both precisions.
#include "rk_launch.cuh"

namespace rk {
RK_INSTANTIATE_LENGTH(8)
}  // namespace rk
