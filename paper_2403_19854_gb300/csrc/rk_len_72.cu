// Pass kernels for lines of 72 nodes, both precisions.
#include "rk_launch.cuh"

namespace rk {
RK_INSTANTIATE_LENGTH(72)
}  // namespace rk
