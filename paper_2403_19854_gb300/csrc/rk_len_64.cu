// Pass kernels for lines of 64 nodes, both precisions.
#include "rk_launch.cuh"

namespace rk {
RK_INSTANTIATE_LENGTH(64)
}  // namespace rk
