// Pass kernels for lines of 32 nodes, both precisions.
#include "rk_launch.cuh"

namespace rk {
RK_INSTANTIATE_LENGTH(32)
}  // namespace rk
