// Pass kernels for lines of 36 nodes, both precisions.
#include "rk_launch.cuh"

namespace rk {
RK_INSTANTIATE_LENGTH(36)
}  // namespace rk
