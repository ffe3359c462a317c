// Pass kernels for lines of 128 nodes, both precisions.
#include "rk_launch.cuh"

namespace rk {
RK_INSTANTIATE_LENGTH(128)
}  // namespace rk
