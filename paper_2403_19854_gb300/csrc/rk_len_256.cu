// Pass kernels for lines of 256 nodes, both precisions.
#include "rk_launch.cuh"

namespace rk {
RK_INSTANTIATE_LENGTH(256)
}  // namespace rk
